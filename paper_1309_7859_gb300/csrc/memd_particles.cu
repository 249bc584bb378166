// memd_particles.cu -- particle kernels of MEMD on sm_103a.
//
//   fold / quantise positions into the fixed-point frame of the lattice
//   cloud-in-cell vertex charges (Sec. IV, linear interpolation, one cell)
//   half kick + drift + charge transfer onto the crossed links (Eq. 20, j)
//   application of the transfers to D and to the exact int64 ledger
//   force gather F = qE with the self-energy (Sec. III) and dipole (Sec. V)
//   corrections, the Langevin force and the second half kick
//
// Built with -fmad=false: positions decide integer cell indices, so every
// position update is two IEEE roundings (a product, then a sum), never a
// fused multiply-add.
#include "memd_internal.cuh"

namespace memd {

namespace {

constexpr int kThreads = 128;
constexpr int kRedThreads = 256;
constexpr int kRedBlocks = 2 * 152;

inline unsigned blocks_for(int64_t n, int t = kThreads) {
  int64_t b = (n + t - 1) / t;
  return (unsigned)(b < 1 ? 1 : b);
}

// ------------------------------------------------------------ fixed point
// Fold x into [0, L) counting images; x == L after rounding maps to 0 in the
// next image.
__device__ inline void fold(double L, double& x, int& img) {
  const double fl = floor(__ddiv_rn(x, L));
  double y = __dsub_rn(x, __dmul_rn(fl, L));
  int k = (int)fl;
  if (y < 0.0) {
    y = __dadd_rn(y, L);
    k -= 1;
  }
  if (y >= L) {
    y = 0.0;
    k += 1;
  }
  x = y;
  img += k;
}

// cell c = floor(x / a) and sub-cell step f = floor((x/a - c) S)
__device__ inline void quantize(const Mesh& m, int d, double x, int& c, int& f) {
  const double u = __ddiv_rn(x, m.a);
  const double cu = floor(u);
  if (cu >= (double)m.n[d]) {
    c = m.n[d] - 1;
    f = (int)kS - 1;
    return;
  }
  if (cu < 0.0) {
    c = 0;
    f = 0;
    return;
  }
  c = (int)cu;
  f = (int)floor(__dmul_rn(__dsub_rn(u, cu), (double)kS));
}

__device__ inline long long wgt(int f, int a) { return a ? (long long)f : (long long)(kS - f); }

__device__ inline int64_t link_index(const Mesh& m, int d, int ci, int cj, int ck) {
  return (int64_t)d * m.V + vindex(m, wrapi(ci, m.n[0]), wrapi(cj, m.n[1]), wrapi(ck, m.n[2]));
}

// warp-aggregated int64 atomic add into a device word
__device__ inline void warp_atomic_add(unsigned long long* addr, long long val) {
  for (int o = 16; o > 0; o >>= 1) val += __shfl_down_sync(0xffffffffu, val, o);
  if ((threadIdx.x & 31) == 0 && val != 0) atomicAdd(addr, (unsigned long long)val);
}

// ------------------------------------------------------------ Philox4x32-10
// Salmon, Moraes, Dror, Shaw (SC'11): ten rounds of two 32x32 -> 64-bit
// products with a Weyl-sequence key schedule.
__device__ inline void philox4x32_10(unsigned c[4], unsigned k0, unsigned k1) {
#pragma unroll
  for (int r = 0; r < 10; ++r) {
    const unsigned lo0 = 0xD2511F53u * c[0], hi0 = __umulhi(0xD2511F53u, c[0]);
    const unsigned lo1 = 0xCD9E8D57u * c[2], hi1 = __umulhi(0xCD9E8D57u, c[2]);
    const unsigned n0 = hi1 ^ c[1] ^ k0;
    const unsigned n2 = hi0 ^ c[3] ^ k1;
    c[0] = n0;
    c[1] = lo1;
    c[2] = n2;
    c[3] = lo0;
    k0 += 0x9E3779B9u;
    k1 += 0xBB67AE85u;
  }
}

__device__ inline double unit_noise(unsigned r) {
  const double u = __dmul_rn(__dadd_rn((double)r, 0.5), 2.3283064365386963e-10);  // 2^-32
  return __dmul_rn(sqrt(3.0), __dsub_rn(__dmul_rn(2.0, u), 1.0));
}

// ---------------------------------------------------------- charge transfer
// Move along axis d from (c0, f0) to (c1, f1) with image change dimg: the
// 4 d-links of the cell change flux by -q (distance) (perpendicular weight);
// a crossed cell face splits the move over the old and the new link.
__device__ inline void deposit_axis(const Mesh& m, int d, int q, int c0, int f0, int c1, int f1,
                                    int dimg, const int cc[3], const int cf[3],
                                    unsigned long long* Tb) {
  const int e1 = (d + 1) % 3, e2 = (d + 2) % 3;
  const int dc = c1 + dimg * m.n[d] - c0;
#pragma unroll
  for (int a2 = 0; a2 < 2; ++a2)
#pragma unroll
    for (int a1 = 0; a1 < 2; ++a1) {
      const long long wp = wgt(cf[e1], a1) * wgt(cf[e2], a2);
      if (wp == 0) continue;
      int at[3] = {cc[0], cc[1], cc[2]};
      at[e1] += a1;
      at[e2] += a2;
      at[d] = c0;
      const int64_t l0 = link_index(m, d, at[0], at[1], at[2]);
      if (dc == 0) {
        const long long t = -(long long)q * (long long)(f1 - f0) * wp;
        if (t) atomicAdd(&Tb[l0], (unsigned long long)t);
      } else if (dc == 1) {
        at[d] = c0 + 1;
        const int64_t l1 = link_index(m, d, at[0], at[1], at[2]);
        const long long t0 = -(long long)q * (long long)(kS - f0) * wp;
        const long long t1 = -(long long)q * (long long)f1 * wp;
        if (t0) atomicAdd(&Tb[l0], (unsigned long long)t0);
        if (t1) atomicAdd(&Tb[l1], (unsigned long long)t1);
      } else {
        at[d] = c0 - 1;
        const int64_t l1 = link_index(m, d, at[0], at[1], at[2]);
        const long long t0 = (long long)q * (long long)f0 * wp;
        const long long t1 = (long long)q * (long long)(kS - f1) * wp;
        if (t0) atomicAdd(&Tb[l0], (unsigned long long)t0);
        if (t1) atomicAdd(&Tb[l1], (unsigned long long)t1);
      }
    }
}

// Move particle p to (xn, kn): axes in the order x, y, z, each with the
// perpendicular weights of the moves made so far.  Returns false (and moves
// nothing) when an axis would cross more than one cell.
__device__ inline bool move_particle(const Mesh& m, Particles P, int64_t p, const double xn[3],
                                     const int kn[3], unsigned long long* Tb, int c1out[3],
                                     int f1out[3]) {
  int c0[3], f0[3], c1[3], f1[3], ko[3];
  for (int d = 0; d < 3; ++d) {
    quantize(m, d, P.x[3 * p + d], c0[d], f0[d]);
    quantize(m, d, xn[d], c1[d], f1[d]);
    ko[d] = P.img[3 * p + d];
    const int dc = c1[d] + (kn[d] - ko[d]) * m.n[d] - c0[d];
    if (dc < -1 || dc > 1) {
      for (int e = 0; e < 3; ++e) {
        c1out[e] = c0[e];
        f1out[e] = f0[e];
      }
      int* mv = P.mv + 6 * p;
      for (int e = 0; e < 3; ++e) {
        mv[e] = c0[e];
        mv[3 + e] = c0[e];
      }
      return false;
    }
  }
  int cc[3] = {c0[0], c0[1], c0[2]}, cf[3] = {f0[0], f0[1], f0[2]};
  const int q = P.q[p];
  for (int d = 0; d < 3; ++d) {
    deposit_axis(m, d, q, c0[d], f0[d], c1[d], f1[d], kn[d] - ko[d], cc, cf, Tb);
    cc[d] = c1[d];
    cf[d] = f1[d];
  }
  for (int d = 0; d < 3; ++d) {
    P.x[3 * p + d] = xn[d];
    P.img[3 * p + d] = kn[d];
    c1out[d] = c1[d];
    f1out[d] = f1[d];
  }
  int* mv = P.mv + 6 * p;
  for (int d = 0; d < 3; ++d) {
    mv[d] = c0[d];
    mv[3 + d] = c1[d];
  }
  return true;
}

__device__ inline void accumulate_dipole(const Mesh& m, int q, const int img[3], const int c[3],
                                         const int f[3], bool active, DevState* ds) {
  for (int d = 0; d < 3; ++d) {
    long long U = ((long long)img[d] * m.n[d] + c[d]) * kS + f[d];
    warp_atomic_add(&ds->Pacc[d], active ? (long long)q * U : 0ll);
  }
}

// ------------------------------------------------------------------ kernels
__global__ void k_fold_init(Mesh m, Particles P, const double* __restrict__ pos,
                            const int* __restrict__ img_in, unsigned int* err) {
  const int64_t p = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (p >= P.n) return;
  for (int d = 0; d < 3; ++d) {
    double x = pos[3 * p + d];
    int k = img_in ? img_in[3 * p + d] : 0;
    if (!(fabs(x) <= 4.0 * m.L[d])) {
      atomicOr(err, kErrNonFinite);
      x = 0.0;
    }
    fold(m.L[d], x, k);
    P.x[3 * p + d] = x;
    P.img[3 * p + d] = k;
  }
}

__global__ void k_cic(Mesh m, Particles P, unsigned long long* __restrict__ Q) {
  const int64_t p = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (p >= P.n) return;
  int c[3], f[3];
  for (int d = 0; d < 3; ++d) quantize(m, d, P.x[3 * p + d], c[d], f[d]);
  const long long q = P.q[p];
  for (int az = 0; az < 2; ++az)
    for (int ay = 0; ay < 2; ++ay)
      for (int ax = 0; ax < 2; ++ax) {
        const long long w = wgt(f[0], ax) * wgt(f[1], ay) * wgt(f[2], az);
        if (w == 0) continue;
        const int64_t v = vindex(m, wrapi(c[0] + ax, m.n[0]), wrapi(c[1] + ay, m.n[1]),
                                 wrapi(c[2] + az, m.n[2]));
        atomicAdd(&Q[v], (unsigned long long)(q * w));
      }
}

__global__ void k_sub_background(int64_t V, long long* __restrict__ Q, long long bg) {
  const int64_t v = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (v < V) Q[v] -= bg;
}

__global__ void k_dipole(Mesh m, Particles P, DevState* ds) {
  const int64_t p = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  const bool active = p < P.n;
  int c[3] = {0, 0, 0}, f[3] = {0, 0, 0}, img[3] = {0, 0, 0};
  int q = 0;
  if (active) {
    q = P.q[p];
    for (int d = 0; d < 3; ++d) {
      quantize(m, d, P.x[3 * p + d], c[d], f[d]);
      img[d] = P.img[3 * p + d];
    }
  }
  accumulate_dipole(m, q, img, c, f, active, ds);
}

// half kick with the stored force, drift, charge transfer, dipole sum
__global__ void __launch_bounds__(kThreads)
    k_kick_drift_deposit(Mesh m, StepParams sp, Particles P, unsigned long long* __restrict__ Tb,
                         DevState* ds) {
  const int64_t p = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  const bool active = p < P.n;
  int c1[3] = {0, 0, 0}, f1[3] = {0, 0, 0}, kn[3] = {0, 0, 0};
  int q = 0;
  if (active) {
    q = P.q[p];
    const double h = __ddiv_rn(0.5 * sp.dt, P.m[p]);
    double xn[3];
    bool ok = true;
    for (int d = 0; d < 3; ++d) {
      const double v = __dadd_rn(P.v[3 * p + d], __dmul_rn(h, P.Ft[3 * p + d]));
      P.v[3 * p + d] = v;
      const double step = __dmul_rn(sp.dt, v);
      if (!(fabs(step) <= 2.0 * m.a)) ok = false;
      xn[d] = __dadd_rn(P.x[3 * p + d], step);
      kn[d] = P.img[3 * p + d];
      if (ok) fold(m.L[d], xn[d], kn[d]);
    }
    if (!ok || !move_particle(m, P, p, xn, kn, Tb, c1, f1)) {
      atomicOr(&ds->err, kErrCellJump);
      for (int d = 0; d < 3; ++d) {
        quantize(m, d, P.x[3 * p + d], c1[d], f1[d]);
        kn[d] = P.img[3 * p + d];
        P.mv[6 * p + d] = c1[d];
        P.mv[6 * p + 3 + d] = c1[d];
      }
    }
  }
  accumulate_dipole(m, q, kn, c1, f1, active, ds);
}

// prescribed move to (pos_new, img_new) with its charge transfer
__global__ void __launch_bounds__(kThreads)
    k_move_deposit(Mesh m, Particles P, const double* __restrict__ pos_new,
                   const int* __restrict__ img_new, unsigned long long* __restrict__ Tb,
                   DevState* ds) {
  const int64_t p = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  const bool active = p < P.n;
  int c1[3] = {0, 0, 0}, f1[3] = {0, 0, 0}, kn[3] = {0, 0, 0};
  int q = 0;
  if (active) {
    q = P.q[p];
    double xn[3];
    bool ok = true;
    for (int d = 0; d < 3; ++d) {
      xn[d] = pos_new[3 * p + d];
      kn[d] = img_new ? img_new[3 * p + d] : 0;
      if (!(fabs(xn[d]) <= 4.0 * m.L[d])) ok = false;
      if (ok) fold(m.L[d], xn[d], kn[d]);
    }
    if (!ok || !move_particle(m, P, p, xn, kn, Tb, c1, f1)) {
      atomicOr(&ds->err, kErrCellJump);
      for (int d = 0; d < 3; ++d) {
        quantize(m, d, P.x[3 * p + d], c1[d], f1[d]);
        kn[d] = P.img[3 * p + d];
        P.mv[6 * p + d] = c1[d];
        P.mv[6 * p + 3 + d] = c1[d];
      }
    }
  }
  accumulate_dipole(m, q, kn, c1, f1, active, ds);
}

// Apply the step's transfers: the first thread to take a link's buffered
// transfer adds it to the ledger exactly and to D scaled by 2^-48 / a^2.
template <typename T>
__global__ void __launch_bounds__(kThreads)
    k_apply(Mesh m, Particles P, unsigned long long* __restrict__ Tb, long long* __restrict__ Lg,
            T* __restrict__ D, double scale) {
  const int64_t p = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (p >= P.n) return;
  const int* mv = P.mv + 6 * p;
  const int c0[3] = {mv[0], mv[1], mv[2]};
  const int c1[3] = {mv[3], mv[4], mv[5]};
  for (int d = 0; d < 3; ++d) {
    const int e1 = (d + 1) % 3, e2 = (d + 2) % 3;
    // perpendicular cells at the time of the move along d: axes before d
    // have moved, axes after d have not
    const int p1 = (e1 < d) ? c1[e1] : c0[e1];
    const int p2 = (e2 < d) ? c1[e2] : c0[e2];
    const int nalong = (c1[d] != c0[d]) ? 2 : 1;
    for (int s = 0; s < nalong; ++s) {
      const int ca = s ? c1[d] : c0[d];
      for (int a2 = 0; a2 < 2; ++a2)
        for (int a1 = 0; a1 < 2; ++a1) {
          int at[3];
          at[d] = ca;
          at[e1] = p1 + a1;
          at[e2] = p2 + a2;
          const int64_t l = link_index(m, d, at[0], at[1], at[2]);
          const long long t = (long long)atomicExch(&Tb[l], 0ull);
          if (t != 0) {
            Lg[l] += t;
            D[l] = D[l] + (T)((double)t * scale);
          }
        }
    }
  }
}

// ------------------------------------------------------------- self energy
// U_self = q^2 / (2 a eps) sum_{r in {0,1}^3} G(r) prod_d c_d(r_d) with
// c(0) = (1-f)^2 + f^2, c(1) = 2 f (1-f); the correction force is +dU/dx.
__device__ inline void self_terms(const StepParams& sp, double a, const int f[3], double q,
                                  double ie_energy, const double ie_dir[3], double& U,
                                  double F3[3]) {
  double c[3][2], dc[3][2];
  for (int d = 0; d < 3; ++d) {
    const double t = (double)f[d] / (double)kS;
    c[d][0] = 1.0 - 2.0 * t + 2.0 * t * t;
    c[d][1] = 2.0 * t - 2.0 * t * t;
    dc[d][0] = 4.0 * t - 2.0;
    dc[d][1] = 2.0 - 4.0 * t;
  }
  double u = 0.0, g0 = 0.0, g1 = 0.0, g2 = 0.0;
  for (int t = 0; t < 8; ++t) {
    const int x = t & 1, y = (t >> 1) & 1, z = (t >> 2) & 1;
    u += sp.G[t] * c[0][x] * c[1][y] * c[2][z];
    g0 += sp.G[t] * dc[0][x] * c[1][y] * c[2][z];
    g1 += sp.G[t] * c[0][x] * dc[1][y] * c[2][z];
    g2 += sp.G[t] * c[0][x] * c[1][y] * dc[2][z];
  }
  const double pre = q * q / (2.0 * a);
  U = pre * ie_energy * u;
  F3[0] = pre * ie_dir[0] * g0 / a;
  F3[1] = pre * ie_dir[1] * g1 / a;
  F3[2] = pre * ie_dir[2] * g2 / a;
}

// GF: mean 1/eps of the 12 cell links for every direction; DIRECT: per
// direction d the weighted mean of 1/eps over the 4 d-links.
__device__ inline void self_ie(const Mesh& m, const double* __restrict__ ie64, const int c[3],
                               const int f[3], int mode, double& ie_cell, double ie_dir[3]) {
  double tot = 0.0;
  for (int d = 0; d < 3; ++d) {
    const int e1 = (d + 1) % 3, e2 = (d + 2) % 3;
    double wd = 0.0;
    for (int a2 = 0; a2 < 2; ++a2)
      for (int a1 = 0; a1 < 2; ++a1) {
        int at[3] = {c[0], c[1], c[2]};
        at[e1] += a1;
        at[e2] += a2;
        const double w = ((double)wgt(f[e1], a1) / (double)kS) * ((double)wgt(f[e2], a2) / (double)kS);
        const double iv = ie64[link_index(m, d, at[0], at[1], at[2])];
        tot += iv;
        wd += iv * w;
      }
    ie_dir[d] = wd;
  }
  ie_cell = tot / 12.0;
  if (mode != 2)
    for (int d = 0; d < 3; ++d) ie_dir[d] = ie_cell;
}

// force gather (Eq. 18 without v x B): E_d from the 4 d-links of the cell
// with the same weights that carry the current, in the field precision T
// the last CTA of the gather closes the update: P of this state becomes the
// reported one, the accumulator is cleared for the next move, and the step
// counter advances (finish == 2)
__device__ inline void finish_update(DevState* ds, int finish) {
  __syncthreads();
  if (threadIdx.x == 0) {
    __threadfence();
    const unsigned t = atomicAdd(&ds->ticket, 1u);
    if (t == gridDim.x - 1) {
      __threadfence();
      for (int d = 0; d < 3; ++d) {
        ds->Plast[d] = (long long)atomicAdd(&ds->Pacc[d], 0ull);
        ds->Pacc[d] = 0ull;
      }
      if (finish == 2) ds->step += 1;
      ds->ticket = 0u;
      __threadfence();
    }
  }
}

template <typename T>
__device__ inline void gather_one(const Mesh& m, const StepParams& sp, Particles P, int64_t p,
                                  const T* __restrict__ D, const T* __restrict__ ie,
                                  const double* __restrict__ ie64, DevState* ds, int kick) {
  int c[3], f[3];
  for (int d = 0; d < 3; ++d) quantize(m, d, P.x[3 * p + d], c[d], f[d]);
  const double q = (double)P.q[p];
  double F[3];
  for (int d = 0; d < 3; ++d) {
    const int e1 = (d + 1) % 3, e2 = (d + 2) % 3;
    T E = T(0);
    for (int a2 = 0; a2 < 2; ++a2)
      for (int a1 = 0; a1 < 2; ++a1) {
        int at[3] = {c[0], c[1], c[2]};
        at[e1] += a1;
        at[e2] += a2;
        const int64_t l = link_index(m, d, at[0], at[1], at[2]);
        const T w = ((T)wgt(f[e1], a1) / (T)kS) * ((T)wgt(f[e2], a2) / (T)kS);
        E = E + D[l] * ie[l] * w;
      }
    F[d] = q * (double)E;
  }
  if (sp.self_mode != 0) {
    double U, Fs[3], ie_cell, ie_dir[3];
    self_ie(m, ie64, c, f, sp.self_mode, ie_cell, ie_dir);
    self_terms(sp, m.a, f, q, ie_cell, ie_dir, U, Fs);
    for (int d = 0; d < 3; ++d) F[d] = F[d] + Fs[d];
  }
  if (sp.dipole_corr) {
    double Pd[3];
    for (int d = 0; d < 3; ++d) Pd[d] = (double)(long long)ds->Pacc[d] * (m.a / (double)kS);
    for (int d = 0; d < 3; ++d) {
      const double MP = sp.Minv[3 * d] * Pd[0] + sp.Minv[3 * d + 1] * Pd[1] + sp.Minv[3 * d + 2] * Pd[2];
      F[d] = F[d] + q * MP / sp.Vbox;
    }
  }
  double Ft[3] = {F[0], F[1], F[2]};
  if (sp.thermo) {
    const long long step = ds->step;
    unsigned ctr[4] = {(unsigned)p, (unsigned)((unsigned long long)p >> 32), (unsigned)step,
                       (unsigned)((unsigned long long)step >> 32)};
    philox4x32_10(ctr, (unsigned)sp.seed, (unsigned)(sp.seed >> 32));
    const double mass = P.m[p];
    const double sig = sqrt(2.0 * sp.gamma * mass * sp.kT / sp.dt);
    for (int d = 0; d < 3; ++d) {
      const double fr = -sp.gamma * mass * P.v[3 * p + d];
      const double fn = sig * unit_noise(ctr[d]);
      Ft[d] = F[d] + (fr + fn);
    }
  }
  for (int d = 0; d < 3; ++d) {
    P.F[3 * p + d] = F[d];
    P.Ft[3 * p + d] = Ft[d];
  }
  if (kick) {
    const double h = __ddiv_rn(0.5 * sp.dt, P.m[p]);
    for (int d = 0; d < 3; ++d) P.v[3 * p + d] = __dadd_rn(P.v[3 * p + d], __dmul_rn(h, Ft[d]));
  }
}

template <typename T>
__global__ void __launch_bounds__(kThreads)
    k_gather(Mesh m, StepParams sp, Particles P, const T* __restrict__ D, const T* __restrict__ ie,
             const double* __restrict__ ie64, DevState* ds, int kick, int finish) {
  const int64_t p = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (p < P.n) gather_one<T>(m, sp, P, p, D, ie, ie64, ds, kick);
  if (finish) finish_update(ds, finish);
}

__global__ void k_step_end(DevState* ds, int advance) {
  if (threadIdx.x == 0 && blockIdx.x == 0) {
    for (int d = 0; d < 3; ++d) {
      ds->Plast[d] = (long long)ds->Pacc[d];
      ds->Pacc[d] = 0ull;
    }
    if (advance) ds->step += 1;
  }
}

__device__ inline double block_sum(double x, double* sh) {
  for (int o = 16; o > 0; o >>= 1) x += __shfl_down_sync(0xffffffffu, x, o);
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  if (lane == 0) sh[w] = x;
  __syncthreads();
  double r = 0.0;
  if (threadIdx.x == 0)
    for (int t = 0; t < (int)(blockDim.x >> 5); ++t) r += sh[t];
  __syncthreads();
  return r;
}

__global__ void __launch_bounds__(kRedThreads)
    k_particle_energy(Mesh m, StepParams sp, Particles P, const double* __restrict__ ie64,
                      double* part_ke, double* part_self) {
  __shared__ double sh[kRedThreads / 32];
  double ke = 0.0, se = 0.0;
  for (int64_t p = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; p < P.n;
       p += (int64_t)gridDim.x * blockDim.x) {
    for (int d = 0; d < 3; ++d) ke += 0.5 * P.m[p] * P.v[3 * p + d] * P.v[3 * p + d];
    if (sp.self_mode != 0) {
      int c[3], f[3];
      for (int d = 0; d < 3; ++d) quantize(m, d, P.x[3 * p + d], c[d], f[d]);
      double U, Fs[3], ie_cell, ie_dir[3];
      self_ie(m, ie64, c, f, sp.self_mode, ie_cell, ie_dir);
      self_terms(sp, m.a, f, (double)P.q[p], ie_cell, ie_dir, U, Fs);
      se += U;
    }
  }
  const double s1 = block_sum(ke, sh);
  const double s2 = block_sum(se, sh);
  if (threadIdx.x == 0) {
    part_ke[blockIdx.x] = s1;
    part_self[blockIdx.x] = s2;
  }
}

}  // namespace

void launch_fold_init(const Mesh& m, Particles p, const double* pos_in, const int* img_in,
                      unsigned int* err, cudaStream_t st) {
  if (p.n > 0) k_fold_init<<<blocks_for(p.n), kThreads, 0, st>>>(m, p, pos_in, img_in, err);
}

void launch_cic(const Mesh& m, Particles p, long long* Q, long long bg, cudaStream_t st) {
  cudaMemsetAsync(Q, 0, sizeof(long long) * m.V, st);
  if (p.n > 0) k_cic<<<blocks_for(p.n), kThreads, 0, st>>>(m, p, (unsigned long long*)Q);
  if (bg != 0) k_sub_background<<<blocks_for(m.V, 256), 256, 0, st>>>(m.V, Q, bg);
}

void launch_dipole(const Mesh& m, Particles p, DevState* ds, cudaStream_t st) {
  cudaMemsetAsync(ds->Pacc, 0, sizeof(ds->Pacc), st);
  if (p.n > 0) k_dipole<<<blocks_for(p.n), kThreads, 0, st>>>(m, p, ds);
}

void launch_kick_drift_deposit(const Mesh& m, const StepParams& sp, Particles p, long long* Tb,
                               DevState* ds, cudaStream_t st) {
  if (p.n > 0)
    k_kick_drift_deposit<<<blocks_for(p.n), kThreads, 0, st>>>(m, sp, p, (unsigned long long*)Tb,
                                                               ds);
}

void launch_move_deposit(const Mesh& m, Particles p, const double* pos_new, const int* img_new,
                         long long* Tb, DevState* ds, cudaStream_t st) {
  if (p.n > 0)
    k_move_deposit<<<blocks_for(p.n), kThreads, 0, st>>>(m, p, pos_new, img_new,
                                                         (unsigned long long*)Tb, ds);
}

void launch_apply(const Mesh& m, int prec, Particles p, long long* Tb, long long* Lg, void* D,
                  double scale, cudaStream_t st) {
  if (p.n <= 0) return;
  if (prec == 1)
    k_apply<float><<<blocks_for(p.n), kThreads, 0, st>>>(m, p, (unsigned long long*)Tb, Lg,
                                                         (float*)D, scale);
  else
    k_apply<double><<<blocks_for(p.n), kThreads, 0, st>>>(m, p, (unsigned long long*)Tb, Lg,
                                                          (double*)D, scale);
}

void launch_gather(const Mesh& m, int prec, const StepParams& sp, Particles p, const void* D,
                   const void* ie, const double* ie64, DevState* ds, int kick, int finish,
                   cudaStream_t st) {
  if (p.n <= 0) {
    if (finish) k_step_end<<<1, 32, 0, st>>>(ds, finish == 2 ? 1 : 0);
    return;
  }
  if (prec == 1)
    k_gather<float><<<blocks_for(p.n), kThreads, 0, st>>>(m, sp, p, (const float*)D,
                                                          (const float*)ie, ie64, ds, kick, finish);
  else
    k_gather<double><<<blocks_for(p.n), kThreads, 0, st>>>(m, sp, p, (const double*)D,
                                                           (const double*)ie, ie64, ds, kick, finish);
}

void launch_step_end(DevState* ds, int advance, cudaStream_t st) {
  k_step_end<<<1, 32, 0, st>>>(ds, advance);
}

void launch_particle_energy(const Mesh& m, const StepParams& sp, Particles p, const double* ie64,
                            double* part_ke, double* part_self, cudaStream_t st) {
  k_particle_energy<<<kRedBlocks, kRedThreads, 0, st>>>(m, sp, p, ie64, part_ke, part_self);
}

}  // namespace memd
