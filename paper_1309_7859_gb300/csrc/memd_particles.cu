// memd_particles.cu -- particle kernels of MEMD on sm_103a.
//
//   fold / quantise positions into the fixed-point frame of the lattice
//   cloud-in-cell vertex charges (Sec. IV, linear interpolation, one cell)
//   half kick + drift + charge transfer onto the crossed links (Eq. 20, j)
//   application of the transfers to D and to the exact int64 ledger
//   force gather F = qE with the self-energy (Sec. III) and dipole (Sec. V)
//   corrections, the Langevin force and the second half kick
//
// The step kernels give each particle a quad of 4 lanes: the three axes of
// the move, the four corners of the cell, or the three force components run
// side by side, so the serial FP64 chain and the dependent atomics of one
// particle are split four ways (GB300 has little FP64 throughput per SM and
// these kernels are latency bound).
//
// Built with -fmad=false: positions decide integer cell indices, so every
// position update is two IEEE roundings (a product, then a sum), never a
// fused multiply-add.
#include "memd_internal.cuh"
#include "memd_rows.cuh"
#include "memd_site.cuh"

namespace memd {

namespace {

constexpr int kThreads = 128;
constexpr int kQuadThreads = 128;  // at most 32 particles per CTA in the quad kernels
constexpr int kRedThreads = 256;
constexpr int kRedBlocks = 2 * 152;

inline unsigned blocks_for(int64_t n, int t = kThreads) {
  int64_t b = (n + t - 1) / t;
  return (unsigned)(b < 1 ? 1 : b);
}

// CTA size of the quad kernels: small systems use small CTAs so that their
// FP64-heavy lanes spread over all 152 SMs instead of a few
inline int quad_threads(int64_t n) {
  const int64_t want = (4 * n + 2 * 152 - 1) / (2 * 152);
  int t = (int)((want + 31) / 32 * 32);
  return t < 32 ? 32 : (t > kQuadThreads ? kQuadThreads : t);
}

// ------------------------------------------------------------ fixed point
// Sec. V periodic stitching: shift by whole box lengths into [0, L); a sum
// that rounds up to L starts the next image.  Callers bound |x| by a few L.
__device__ inline void fold(double L, double& x, int& img) {
  double y = x;
  int k = 0;
  while (y >= L) {
    y = __dsub_rn(y, L);
    ++k;
  }
  while (y < 0.0) {
    y = __dadd_rn(y, L);
    --k;
  }
  if (y >= L) {
    y = 0.0;
    ++k;
  }
  x = y;
  img += k;
}

// cell c = floor(x / a) and sub-cell step f = floor((x/a - c) S).  When a is
// a power of two, x / a, x / a - c and the scaling by S are all exact, so
// floor(x S / a) = c S + f holds both in one rounding-free product.
__device__ inline void quantize(const Mesh& m, int d, double x, int& c, int& f) {
  if (m.a_pow2) {
    const long long W = __double2ll_rd(__dmul_rn(x, m.inv_aS));
    const long long cw = W >> kWBits;  // floor(W / S)
    if (cw >= (long long)m.n[d]) {
      c = m.n[d] - 1;
      f = (int)kS - 1;
    } else if (cw < 0) {
      c = 0;
      f = 0;
    } else {
      c = (int)cw;
      f = (int)(W & (long long)(kS - 1));
    }
    return;
  }
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

// periodic wrap of a cell index in [-n, 2n): the step kernels only ever
// look one cell beyond a quantised cell, so no integer division is needed
__device__ inline int wrap1(int i, int n) { return i < 0 ? i + n : (i >= n ? i - n : i); }

// the vertex a link leaves (its cell coordinates wrapped once)
__device__ inline int64_t link_vertex(const Mesh& m, int ci, int cj, int ck) {
  return vindex(m, wrap1(ci, m.n[0]), wrap1(cj, m.n[1]), wrap1(ck, m.n[2]));
}

__device__ inline int64_t link_index(const Mesh& m, int d, int ci, int cj, int ck) {
  return (int64_t)d * m.V + link_vertex(m, ci, cj, ck);
}

// warp-aggregated int64 atomic add into a device word
__device__ inline void warp_atomic_add(unsigned long long* addr, long long val) {
  for (int o = 16; o > 0; o >>= 1) val += __shfl_down_sync(0xffffffffu, val, o);
  if ((threadIdx.x & 31) == 0 && val != 0) atomicAdd(addr, (unsigned long long)val);
}

// sum over the 8 quads of a warp of a value held by quad lane d (d = 0..2):
// lane d of the warp ends with the warp total for component d
__device__ inline void quad_dipole_add(unsigned long long* Pacc, long long val) {
  for (int o = 16; o >= 4; o >>= 1) val += __shfl_down_sync(0xffffffffu, val, o);
  const int lane = threadIdx.x & 31;
  if (lane < 3 && val != 0) atomicAdd(&Pacc[lane], (unsigned long long)val);
}

// the same sum over a whole CTA (at most kQuadThreads threads, every thread
// calls it, all adding into the same Pacc): one atomic per component and
// CTA instead of one per warp, since the three words share one L2 line and
// their atomics are processed one after another
constexpr int kDipoleWarps = 16;  // CTAs of up to 512 threads
static_assert(kBatchQuadThreads <= 32 * kDipoleWarps && kQuadThreads <= 32 * kDipoleWarps &&
                  kBatchStepThreads <= 32 * kDipoleWarps,
              "cta_dipole_add sizes its table for kDipoleWarps warps");
__device__ inline void cta_dipole_add(unsigned long long* Pacc, long long val) {
  __shared__ long long part[kDipoleWarps][3];
  for (int o = 16; o >= 4; o >>= 1) val += __shfl_down_sync(0xffffffffu, val, o);
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  if (lane < 3) part[warp][lane] = val;
  __syncthreads();
  if (threadIdx.x < 3) {
    long long s = 0;
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) s += part[w][threadIdx.x];
    if (s != 0) atomicAdd(&Pacc[threadIdx.x], (unsigned long long)s);
  }
}

// the same sum with every thread holding all three components (one thread
// per charge)
__device__ inline void cta_dipole_add3(unsigned long long* Pacc, const long long U[3]) {
  __shared__ long long part3[kDipoleWarps][3];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
  for (int e = 0; e < 3; ++e) {
    long long v = U[e];
    for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
    if (lane == 0) part3[warp][e] = v;
  }
  __syncthreads();
  if (threadIdx.x < 3) {
    long long s = 0;
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) s += part3[w][threadIdx.x];
    if (s != 0) atomicAdd(&Pacc[threadIdx.x], (unsigned long long)s);
  }
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

// xi = sqrt(3) (2 u - 1), u = (r + 1/2) 2^-32.  2 u - 1 = k 2^-32 with the
// integer k = 2 r + 1 - 2^32 (|k| < 2^32: converted exactly), and scaling the
// double sqrt(3) by 2^-32 is exact, so xi is the one rounding of k times
// sqrt(3) 2^-32: the same double as rounding sqrt(3) (2 u - 1) after forming
// 2 u - 1 exactly, with one conversion and one product on the FP64 pipe
__device__ inline double unit_noise(unsigned r) {
  const long long k = 2 * (long long)r + 1 - (1ll << 32);
  return __dmul_rn(__ll2double_rn(k), 0x1.bb67ae8584caap-32);  // sqrt(3) 2^-32
}

// ---------------------------------------------------------- charge transfer
// Move along axis d from (c0, f0) to (c1, f1), dc = c1 - c0 + dimg N in
// {-1, 0, 1}: the 4 d-links of the cell change flux by -q (distance moved)
// (perpendicular weight); a crossed cell face splits the move over the old
// and the new link.  Perpendicular weights are those of the moves made so
// far (axes before d at their new cells, axes after d at their old ones).
__device__ inline int sel3(int d, int a, int b, int c) { return d == 0 ? a : (d == 1 ? b : c); }

// cmV: the layout of Tb (tw_index)
__device__ inline void deposit_axis(const Mesh& m, int d, int q, int c0, int f0, int f1, int dc,
                                    const int cc[3], const int cf[3],
                                    unsigned long long* __restrict__ Tb, int64_t cmV = 0) {
  // axis d is the lane's own (a run-time value): select sizes, strides and
  // perpendicular coordinates instead of indexing arrays with it
  const int e1 = d == 2 ? 0 : d + 1, e2 = d == 0 ? 2 : d - 1;
  const int64_t st[3] = {1, (int64_t)m.n[0], (int64_t)m.n[0] * m.n[1]};
  const int nd = sel3(d, m.n[0], m.n[1], m.n[2]);
  const int n1 = sel3(e1, m.n[0], m.n[1], m.n[2]), n2 = sel3(e2, m.n[0], m.n[1], m.n[2]);
  const int64_t sd = d == 0 ? st[0] : (d == 1 ? st[1] : st[2]);
  const int64_t s1 = e1 == 0 ? st[0] : (e1 == 1 ? st[1] : st[2]);
  const int64_t s2 = e2 == 0 ? st[0] : (e2 == 1 ? st[1] : st[2]);
  const int v0 = sel3(e1, cc[0], cc[1], cc[2]), w0 = sel3(e2, cc[0], cc[1], cc[2]);
  const int fv = sel3(e1, cf[0], cf[1], cf[2]), fw = sel3(e2, cf[0], cf[1], cf[2]);
  // vertex indices of the old and new cell along d (the link's pair is
  // tl_pair(d, vertex))
  const int64_t u0 = (int64_t)wrap1(c0, nd) * sd;
  const int64_t u1 = (int64_t)wrap1(c0 + dc, nd) * sd;
#pragma unroll
  for (int a2 = 0; a2 < 2; ++a2)
#pragma unroll
    for (int a1 = 0; a1 < 2; ++a1) {
      const long long wp = wgt(fv, a1) * wgt(fw, a2);
      if (wp == 0) continue;
      const int64_t perp = (int64_t)wrap1(v0 + a1, n1) * s1 + (int64_t)wrap1(w0 + a2, n2) * s2;
      const int64_t l0 = u0 + perp;
      if (dc == 0) {
        const long long t = -(long long)q * (long long)(f1 - f0) * wp;
        if (t) red_add_hint(&Tb[tw_index(d, l0, cmV)], (unsigned long long)t, l2_policy_last());
      } else if (dc == 1) {
        const int64_t l1 = u1 + perp;
        const long long t0 = -(long long)q * (long long)(kS - f0) * wp;
        const long long t1 = -(long long)q * (long long)f1 * wp;
        if (t0) red_add_hint(&Tb[tw_index(d, l0, cmV)], (unsigned long long)t0, l2_policy_last());
        if (t1) red_add_hint(&Tb[tw_index(d, l1, cmV)], (unsigned long long)t1, l2_policy_last());
      } else {
        const int64_t l1 = u1 + perp;
        const long long t0 = (long long)q * (long long)f0 * wp;
        const long long t1 = (long long)q * (long long)(kS - f1) * wp;
        if (t0) red_add_hint(&Tb[tw_index(d, l0, cmV)], (unsigned long long)t0, l2_policy_last());
        if (t1) red_add_hint(&Tb[tw_index(d, l1, cmV)], (unsigned long long)t1, l2_policy_last());
      }
    }
}

// Quad lane d (< 3) holds axis d of particle p: its old position x, image
// ko, and the proposed new position xn / image kn (already folded).  The
// quad exchanges the quantised coordinates, deposits one axis per lane and
// commits the move, or leaves the particle where it was (ok == false) when
// some axis would cross more than one cell.  Every lane of the warp must
// call this; inactive lanes pass active = false.  Returns the lane's term of
// the dipole sum (valence times the unfolded fixed-point coordinate along d;
// 0 for lane 3 and inactive lanes), which the caller adds into Pacc.
// pf_ie (optional, element size pf_es): 1/eps in the field precision; the
// links of the cell the charge ends in, which the gather reads next, and the
// charge's mass, valence and noise amplitude are then prefetched into L2.
__device__ inline long long quad_move(const Mesh& m, Particles P, int64_t p, int d, bool active,
                                      double x, int ko, double xn, int kn, bool ok_in,
                                      unsigned long long* __restrict__ Tb, DevState* ds,
                                      const char* pf_ie = nullptr, int pf_es = 0,
                                      int64_t cmV = 0) {
  const unsigned full = 0xffffffffu;
  const int lane = threadIdx.x & 31, base = lane & ~3;
  int c0 = 0, f0 = 0, c1 = 0, f1 = 0, dc = 0;
  bool ok = ok_in;
  if (active && d < 3) {
    quantize(m, d, x, c0, f0);
    quantize(m, d, xn, c1, f1);
    dc = c1 + (kn - ko) * m.n[d] - c0;
    if (dc < -1 || dc > 1) ok = false;
  } else {
    ok = true;
  }
  // all three axes must be valid for the particle to move
  const bool all_ok = ((__ballot_sync(full, ok) >> base) & 0xfu) == 0xfu;
  int C0[3], F0[3], C1[3], F1[3];
#pragma unroll
  for (int e = 0; e < 3; ++e) {
    C0[e] = __shfl_sync(full, c0, base + e);
    F0[e] = __shfl_sync(full, f0, base + e);
    C1[e] = __shfl_sync(full, c1, base + e);
    F1[e] = __shfl_sync(full, f1, base + e);
  }
  if (pf_ie && active) {
    // quad lane d holds corner (d & 1, d >> 1): its three links of the final cell
    const int a1 = d & 1, a2 = d >> 1;
#pragma unroll
    for (int e = 0; e < 3; ++e) {
      const int e1 = (e + 1) % 3, e2 = (e + 2) % 3;
      int at[3] = {all_ok ? C1[0] : C0[0], all_ok ? C1[1] : C0[1], all_ok ? C1[2] : C0[2]};
      at[e1] += a1;
      at[e2] += a2;
      const char* a = pf_ie + link_index(m, e, at[0], at[1], at[2]) * pf_es;
      asm volatile("prefetch.global.L2 [%0];" ::"l"(a));
    }
    if (d == 0) {
      asm volatile("prefetch.global.L2 [%0];" ::"l"(P.gm + p));
      asm volatile("prefetch.global.L2 [%0];" ::"l"(P.sig + p));
      asm volatile("prefetch.global.L2 [%0];" ::"l"(P.q + p));
    }
  }
  long long U = 0;
  if (active && d < 3) {
    int* mv = P.mv + kMoveInts * p;
    if (all_ok) {
      int cc[3], cf[3];
#pragma unroll
      for (int e = 0; e < 3; ++e) {
        cc[e] = (e < d) ? C1[e] : C0[e];
        cf[e] = (e < d) ? F1[e] : F0[e];
      }
      deposit_axis(m, d, P.q[p], c0, f0, f1, dc, cc, cf, Tb, cmV);
      P.x[3 * p + d] = xn;
      P.img[3 * p + d] = kn;
      mv[d] = c0;
      mv[3 + d] = c1;
      mv[6 + d] = f1;
      U = ((long long)kn * m.n[d] + c1) * kS + f1;
    } else {
      mv[d] = c0;
      mv[3 + d] = c0;
      mv[6 + d] = f0;
      U = ((long long)ko * m.n[d] + c0) * kS + f0;
      if (d == 0) atomicOr(&ds->err, kErrCellJump);
    }
    U *= (long long)P.q[p];
  }
  return U;
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
        const int64_t v = vindex(m, wrap1(c[0] + ax, m.n[0]), wrap1(c[1] + ay, m.n[1]),
                                 wrap1(c[2] + az, m.n[2]));
        atomicAdd(&Q[v], (unsigned long long)(q * w));
      }
}

// cloud-in-cell density of |q| (the salt content) at the vertices, int64 in
// units of e 2^-48
__global__ void k_cic_abs(Mesh m, Particles P, unsigned long long* __restrict__ Q) {
  const int64_t p = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (p >= P.n) return;
  int c[3], f[3];
  for (int d = 0; d < 3; ++d) quantize(m, d, P.x[3 * p + d], c[d], f[d]);
  const long long aq = P.q[p] < 0 ? -(long long)P.q[p] : (long long)P.q[p];
  for (int az = 0; az < 2; ++az)
    for (int ay = 0; ay < 2; ++ay)
      for (int ax = 0; ax < 2; ++ax) {
        const long long w = wgt(f[0], ax) * wgt(f[1], ay) * wgt(f[2], az);
        if (w == 0) continue;
        const int64_t v = vindex(m, wrap1(c[0] + ax, m.n[0]), wrap1(c[1] + ay, m.n[1]),
                                 wrap1(c[2] + az, m.n[2]));
        atomicAdd(&Q[v], (unsigned long long)(aq * w));
      }
}

__global__ void k_sub_background(int64_t V, long long* __restrict__ Q, long long bg) {
  const int64_t v = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (v < V) Q[v] -= bg;
}

__global__ void k_dipole(Mesh m, Particles P, DevState* ds) {
  const int64_t p = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  for (int d = 0; d < 3; ++d) {
    long long U = 0;
    if (p < P.n) {
      int c, f;
      quantize(m, d, P.x[3 * p + d], c, f);
      U = (long long)P.q[p] * (((long long)P.img[3 * p + d] * m.n[d] + c) * kS + f);
    }
    warp_atomic_add(&ds->Pacc[d], U);
  }
}

__global__ void k_particle_constants(StepParams sp, Particles P) {
  const int64_t p = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (p >= P.n) return;
  const double mass = P.m[p];
  P.h[p] = __ddiv_rn(0.5 * sp.dt, mass);
  if (sp.thermo) {
    P.sig[p] = sqrt(2.0 * sp.gamma * mass * sp.kT / sp.dt);
    P.gm[p] = __dmul_rn(-sp.gamma, mass);  // the friction's first product, (-gamma) m
  }
}

// half kick with the stored force, drift, charge transfer; g is the
// thread's index within its system; returns the lane's dipole term
__device__ __forceinline__ long long deposit_body(const Mesh& m, const StepParams& sp, Particles P,
                                             unsigned long long* __restrict__ Tb, DevState* ds,
                                             int64_t g, const char* pf_ie = nullptr,
                                             int pf_es = 0, int64_t cmV = 0) {
  const int64_t p = g >> 2;
  const int d = (int)(g & 3);
  const bool active = p < P.n;
  double x = 0.0, xn = 0.0;
  int ko = 0, kn = 0;
  bool ok = true;
  if (active && d < 3) {
    const double v = __dadd_rn(P.v[3 * p + d], __dmul_rn(P.h[p], P.Ft[3 * p + d]));
    P.v[3 * p + d] = v;
    const double step = __dmul_rn(sp.dt, v);
    x = P.x[3 * p + d];
    ko = P.img[3 * p + d];
    kn = ko;
    xn = x;
    if (fabs(step) <= 2.0 * m.a) {
      xn = __dadd_rn(x, step);
      fold(m.L[d], xn, kn);
    } else {
      ok = false;
    }
  }
  return quad_move(m, P, p, d, active, x, ko, xn, kn, ok, Tb, ds, pf_ie, pf_es, cmV);
}

// One thread per charge: the half kick, drift and charge transfer of
// deposit_body and quad_move with the same expressions, the three axes in
// turn.  Sets U to the dipole terms (valence times the unfolded fixed-point
// coordinate of each axis; 0 for a thread past the last charge).  For large
// charge counts: a warp then moves 32 charges an instruction instead of 8,
// with no exchange of cells between lanes.
__device__ __forceinline__ void deposit_wide(const Mesh& m, const StepParams& sp, Particles P,
                                             unsigned long long* __restrict__ Tb, DevState* ds,
                                             int64_t p, long long U[3]) {
  U[0] = U[1] = U[2] = 0;
  if (p >= P.n) return;
  const double h = P.h[p];
  const int q = P.q[p];
  double x[3], xn[3];
  int ko[3], kn[3];
  bool ok = true;
#pragma unroll
  for (int d = 0; d < 3; ++d) {
    const double v = __dadd_rn(P.v[3 * p + d], __dmul_rn(h, P.Ft[3 * p + d]));
    P.v[3 * p + d] = v;
    const double step = __dmul_rn(sp.dt, v);
    x[d] = P.x[3 * p + d];
    ko[d] = P.img[3 * p + d];
    kn[d] = ko[d];
    xn[d] = x[d];
    if (fabs(step) <= 2.0 * m.a) {
      xn[d] = __dadd_rn(x[d], step);
    } else {
      ok = false;
    }
  }
  int c0[3], f0[3], c1[3], f1[3], dc[3];
#pragma unroll
  for (int d = 0; d < 3; ++d) {
    quantize(m, d, x[d], c0[d], f0[d]);
    // With a power-of-two spacing the product x S / a is exact, so xn lies in
    // [0, L) exactly when 0 <= floor(xn S / a) < n S: the quantised value then
    // is the cell and step of the folded position, and the fold's FP64
    // comparisons are skipped (GB300's FP64 pipe is narrow).  Otherwise fold
    // and quantise as the other kernels do; the results are the same.
    bool inside = false;
    if (m.a_pow2) {
      const long long W = __double2ll_rd(__dmul_rn(xn[d], m.inv_aS));
      if (W >= 0 && W < (long long)m.n[d] * kS) {
        inside = true;
        c1[d] = (int)(W >> kWBits);
        f1[d] = (int)(W & (kS - 1));
      }
    }
    if (!inside) {
      fold(m.L[d], xn[d], kn[d]);
      quantize(m, d, xn[d], c1[d], f1[d]);
    }
    dc[d] = c1[d] + (kn[d] - ko[d]) * m.n[d] - c0[d];
    if (dc[d] < -1 || dc[d] > 1) ok = false;
  }
  int* mv = P.mv + kMoveInts * p;
  if (ok) {
#pragma unroll
    for (int d = 0; d < 3; ++d) {
      // perpendicular weights of the moves made so far
      int cc[3], cf[3];
#pragma unroll
      for (int e = 0; e < 3; ++e) {
        cc[e] = (e < d) ? c1[e] : c0[e];
        cf[e] = (e < d) ? f1[e] : f0[e];
      }
      deposit_axis(m, d, q, c0[d], f0[d], f1[d], dc[d], cc, cf, Tb);
      P.x[3 * p + d] = xn[d];
      P.img[3 * p + d] = kn[d];
      mv[d] = c0[d];
      mv[3 + d] = c1[d];
      mv[6 + d] = f1[d];
      U[d] = (((long long)kn[d] * m.n[d] + c1[d]) * kS + f1[d]) * (long long)q;
    }
  } else {
#pragma unroll
    for (int d = 0; d < 3; ++d) {
      mv[d] = c0[d];
      mv[3 + d] = c0[d];
      mv[6 + d] = f0[d];
      U[d] = (((long long)ko[d] * m.n[d] + c0[d]) * kS + f0[d]) * (long long)q;
    }
    atomicOr(&ds->err, kErrCellJump);
  }
}

__global__ void __launch_bounds__(kWideThreads)
    k_deposit_wide(const __grid_constant__ Mesh m, const __grid_constant__ StepParams sp,
                   Particles P, unsigned long long* __restrict__ Tb, DevState* ds) {
  long long U[3];
  deposit_wide(m, sp, P, Tb, ds, blockIdx.x * (int64_t)blockDim.x + threadIdx.x, U);
  cta_dipole_add3(ds->Pacc, U);
}

__global__ void __launch_bounds__(kQuadThreads)
    k_kick_drift_deposit(const __grid_constant__ Mesh m, const __grid_constant__ StepParams sp,
                         Particles P, unsigned long long* __restrict__ Tb,
                         DevState* ds) {
  cta_dipole_add(ds->Pacc,
                 deposit_body(m, sp, P, Tb, ds, blockIdx.x * (int64_t)blockDim.x + threadIdx.x));
}

// prescribed move to (pos_new, img_new) with its charge transfer
__global__ void __launch_bounds__(kQuadThreads)
    k_move_deposit(const __grid_constant__ Mesh m, Particles P, const double* __restrict__ pos_new,
                   const int* __restrict__ img_new, unsigned long long* __restrict__ Tb,
                   DevState* ds) {
  const int64_t g = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  const int64_t p = g >> 2;
  const int d = (int)(g & 3);
  const bool active = p < P.n;
  double x = 0.0, xn = 0.0;
  int ko = 0, kn = 0;
  bool ok = true;
  if (active && d < 3) {
    x = P.x[3 * p + d];
    ko = P.img[3 * p + d];
    xn = pos_new[3 * p + d];
    kn = img_new ? img_new[3 * p + d] : 0;
    if (fabs(xn) <= 4.0 * m.L[d])
      fold(m.L[d], xn, kn);
    else
      ok = false;
  }
  cta_dipole_add(ds->Pacc, quad_move(m, P, p, d, active, x, ko, xn, kn, ok, Tb, ds));
}

// Apply the step's transfers: the first lane to take a link's buffered
// transfer adds it to the ledger exactly and to D scaled by 2^-48 / a^2.
// Quad lane c handles corner (c & 1, c >> 1) of every axis and both cells of
// a crossed face; its exchanges are issued together.
template <typename T>
__device__ __forceinline__ void apply_body(const Mesh& m, Particles P,
                                           unsigned long long* __restrict__ Tb,
                                           long long* __restrict__ Lg, T* __restrict__ D,
                                           double scale, int64_t g, int64_t cmV = 0) {
  const int64_t p = g >> 2;
  if (p >= P.n) return;
  const int corner = (int)(g & 3);
  const int a1 = corner & 1, a2 = corner >> 1;
  // the move record may have been written in this launch by another CTA
  // (single-launch batch step): read through L2
  const int* mv = P.mv + kMoveInts * p;
  const int c0[3] = {__ldcg(mv), __ldcg(mv + 1), __ldcg(mv + 2)};
  const int c1[3] = {__ldcg(mv + 3), __ldcg(mv + 4), __ldcg(mv + 5)};
  // slot 2d: the d-link at the old cell along d; slot 2d+1: at the new
  // cell, when the move crossed a face; v: the vertex the link leaves
  int64_t v[6];
  bool has[6];
#pragma unroll
  for (int d = 0; d < 3; ++d) {
    const int e1 = (d + 1) % 3, e2 = (d + 2) % 3;
    // perpendicular cells at the time of the move along d: axes before d
    // have moved, axes after d have not
    const int p1 = (e1 < d) ? c1[e1] : c0[e1];
    const int p2 = (e2 < d) ? c1[e2] : c0[e2];
    int at[3];
    at[e1] = p1 + a1;
    at[e2] = p2 + a2;
    at[d] = c0[d];
    v[2 * d] = link_vertex(m, at[0], at[1], at[2]);
    has[2 * d] = true;
    at[d] = c1[d];
    v[2 * d + 1] = link_vertex(m, at[0], at[1], at[2]);
    has[2 * d + 1] = c1[d] != c0[d];
  }
  // the transfer and ledger words stay in L2 for the gather's ledger reads
  const unsigned long long pol = l2_policy_last();
  long long t[6];
#pragma unroll
  for (int s = 0; s < 6; ++s)
    t[s] = has[s] ? (long long)exch_hint(&Tb[tw_index(s >> 1, v[s], cmV)], 0ull, pol) : 0ll;
  // only the lane that took a link's transfer adds it, so each reduction
  // below is the one addition to its word in this kernel: exact for the
  // ledger, D + x rounded once for the field
#pragma unroll
  for (int s = 0; s < 6; ++s)
    if (t[s] != 0) {
      red_add_hint((unsigned long long*)&Lg[kLT * tl_pair(s >> 1, v[s])], (unsigned long long)t[s],
                   pol);
      atomicAdd(&D[(int64_t)(s >> 1) * m.V + v[s]], (T)((double)t[s] * scale));
    }
}

template <typename T>
__global__ void __launch_bounds__(kQuadThreads)
    k_apply(const __grid_constant__ Mesh m, Particles P, unsigned long long* __restrict__ Tb, long long* __restrict__ Lg,
            T* __restrict__ D, double scale, int64_t cmV) {
  apply_body<T>(m, P, Tb, Lg, D, scale, blockIdx.x * (int64_t)blockDim.x + threadIdx.x, cmV);
}

// Dense form of the same: every link pair of [l0, l1) once (pair 3 v + d
// is link (d, v), field index d V + v), each non-zero transfer word added to
// the ledger and, scaled, to D, then cleared.  Each word gets the one
// addition the sparse form gives it, so D + x is rounded once the same way.
// A link's transfer and ledger words are one 16-byte pair (read and written
// as a vector when the allocation is 16-byte aligned: a caller's allocator
// need not align it; else word by word).
__device__ inline int64_t pair_field_index(int64_t w, int64_t V) {
  const int64_t v = w / 3;
  return (w - 3 * v) * V + v;
}
template <typename T>
__device__ __forceinline__ void apply_word(long long* __restrict__ Tb, long long* __restrict__ Lg,
                                           T* __restrict__ D, double scale, int64_t w, int64_t V) {
  const long long t = Tb[kLT * w];
  if (t != 0) {
    const int64_t l = pair_field_index(w, V);
    Tb[kLT * w] = 0;
    Lg[kLT * w] += t;
    D[l] = D[l] + (T)((double)t * scale);
  }
}

// a CTA's range is kApplyPairs links a thread; every load (the pairs, then
// D of the non-zero ones) is issued before any store, so a thread waits for
// two round trips, not two per link
template <typename T>
__device__ __forceinline__ void apply_dense_range(long long* __restrict__ Tb,
                                                  long long* __restrict__ Lg, T* __restrict__ D,
                                                  double scale, int64_t l0, int64_t l1,
                                                  int64_t V) {
  if (reinterpret_cast<uintptr_t>(Tb) & 15) {
    for (int64_t l = l0 + threadIdx.x; l < l1; l += blockDim.x)
      apply_word<T>(Tb, Lg, D, scale, l, V);
    return;
  }
  longlong2* TL = reinterpret_cast<longlong2*>(Tb);  // (transfer, ledger) of each link
  longlong2 tl[2 * kApplyPairs];
  T dv[2 * kApplyPairs];
  int64_t w[2 * kApplyPairs];
#pragma unroll
  for (int j = 0; j < 2 * kApplyPairs; ++j) {
    w[j] = l0 + threadIdx.x + (int64_t)j * blockDim.x;
    tl[j] = w[j] < l1 ? __ldcs(TL + w[j]) : make_longlong2(0, 0);
  }
#pragma unroll
  for (int j = 0; j < 2 * kApplyPairs; ++j)
    dv[j] = tl[j].x != 0 ? D[pair_field_index(w[j], V)] : T(0);
#pragma unroll
  for (int j = 0; j < 2 * kApplyPairs; ++j)
    if (tl[j].x != 0) {
      TL[w[j]] = make_longlong2(0, tl[j].y + tl[j].x);
      D[pair_field_index(w[j], V)] = dv[j] + (T)((double)tl[j].x * scale);
    }
}

template <typename T>
__global__ void __launch_bounds__(kApplyThreads)
    k_apply_dense(int64_t nl, long long* __restrict__ Tb, long long* __restrict__ Lg,
                  T* __restrict__ D, double scale) {
  const int64_t l0 = (int64_t)blockIdx.x * kApplyChunk;
  apply_dense_range<T>(Tb, Lg, D, scale, l0, l0 + kApplyChunk < nl ? l0 + kApplyChunk : nl,
                       nl / 3);
}

// ------------------------------------------------------------- self energy
// U_self = q^2 / (2 a eps) sum_{r in {0,1}^3} G(r) prod_d c_d(r_d) with
// c(0) = (1-f)^2 + f^2, c(1) = 2 f (1-f); the correction force is +dU/dx.
// R is the arithmetic type of the force terms: double with FP64 fields,
// float with FP32 fields.
template <typename R>
struct SelfC {
  R c[3][2], dc[3][2];
};

// c(1) = 2 t (1 - t), c(0) = 1 - c(1), dc/dt = +-(4 t - 2), t = f / S
template <typename R>
__device__ inline SelfC<R> self_coeffs(const int f[3]) {
  SelfC<R> s;
#pragma unroll
  for (int d = 0; d < 3; ++d) {
    const R t = (R)f[d] * (R(1) / (R)kS);
    const R u = R(2) * (t * (R(1) - t));
    s.c[d][0] = R(1) - u;
    s.c[d][1] = u;
    s.dc[d][0] = R(4) * t - R(2);
    s.dc[d][1] = -s.dc[d][0];
  }
  return s;
}

// step constants in the force precision R
template <typename R>
__device__ inline R sp_G(const StepParams& sp, int i);
template <>
__device__ inline double sp_G<double>(const StepParams& sp, int i) { return sp.G[i]; }
template <>
__device__ inline float sp_G<float>(const StepParams& sp, int i) { return sp.Gf[i]; }
template <typename R>
__device__ inline R sp_Mdip(const StepParams& sp, int i);
template <>
__device__ inline double sp_Mdip<double>(const StepParams& sp, int i) { return sp.Mdip[i]; }
template <>
__device__ inline float sp_Mdip<float>(const StepParams& sp, int i) { return sp.Mdipf[i]; }
template <typename R>
__device__ inline R sp_self_pre(const StepParams& sp);
template <>
__device__ inline double sp_self_pre<double>(const StepParams& sp) { return sp.self_pre; }
template <>
__device__ inline float sp_self_pre<float>(const StepParams& sp) { return sp.self_pref; }

// sum_r G(r) a_x(r_x) a_y(r_y) a_z(r_z) with the derivative factor along
// `dir`, summed axis by axis (x first, then y, then z)
template <typename R>
__device__ inline R self_sum(const StepParams& sp, const SelfC<R>& s, int dir) {
  const R x0 = dir == 0 ? s.dc[0][0] : s.c[0][0], x1 = dir == 0 ? s.dc[0][1] : s.c[0][1];
  const R y0 = dir == 1 ? s.dc[1][0] : s.c[1][0], y1 = dir == 1 ? s.dc[1][1] : s.c[1][1];
  const R z0 = dir == 2 ? s.dc[2][0] : s.c[2][0], z1 = dir == 2 ? s.dc[2][1] : s.c[2][1];
  R sz[2];
#pragma unroll
  for (int z = 0; z < 2; ++z) {
    const R s0 = sp_G<R>(sp, 4 * z) * x0 + sp_G<R>(sp, 4 * z + 1) * x1;
    const R s1 = sp_G<R>(sp, 4 * z + 2) * x0 + sp_G<R>(sp, 4 * z + 3) * x1;
    sz[z] = s0 * y0 + s1 * y1;
  }
  return sz[0] * z0 + sz[1] * z1;
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

// the last CTA of the gather closes the update: P of this state becomes the
// reported one, the accumulator is cleared for the next move, and the step
// counter advances (finish == 2)
// The accumulator was completed by an earlier kernel; what must not be
// overtaken are this kernel's reads of it (and of the step counter), which
// every CTA finishes before its barrier and its acq_rel ticket.
__device__ inline void finish_update(DevState* ds, int finish, unsigned nctas) {
  __syncthreads();
  if (threadIdx.x == 0 && threadIdx.y == 0) {
    unsigned t;
    asm volatile("atom.acq_rel.gpu.global.add.u32 %0, [%1], 1;"
                 : "=r"(t)
                 : "l"(&ds->ticket)
                 : "memory");
    if (t == nctas - 1) {
      const unsigned long long p0 = ds->Pacc[0], p1 = ds->Pacc[1], p2 = ds->Pacc[2];
      ds->Plast[0] = (long long)p0;
      ds->Plast[1] = (long long)p1;
      ds->Plast[2] = (long long)p2;
      ds->Pacc[0] = 0ull;
      ds->Pacc[1] = 0ull;
      ds->Pacc[2] = 0ull;
      if (finish == 2) ds->step += 1;
      ds->ticket = 0u;
    }
  }
}

// Force gather (Eq. 18 without v x B).  Quad lane c loads corner
// (c & 1, c >> 1) of the cell's d-links for the three axes; the quad sums
// E_d = sum D ie w (field precision T) and the 1/eps averages of the self
// term; then lane d < 3 finishes component d: q E_d, the self-energy and
// dipole corrections, the Langevin force and the half kick.
template <typename T>
__device__ __forceinline__ void gather_body(const Mesh& m, const StepParams& sp, int thermo,
                                            double gamma, double kT, Particles P,
                                            const T* __restrict__ D, const T* __restrict__ ie,
                                            const double* __restrict__ ie64, DevState* ds,
                                            int kick, int finish, unsigned nctas, int64_t g,
                                            const long long* __restrict__ Tpend = nullptr,
                                            bool exact32 = false, const long long* pre = nullptr,
                                            bool use_mv = false) {
  const int64_t p = g >> 2;
  const int lane4 = (int)(g & 3);
  const bool active = p < P.n;
  const bool comp = active && lane4 < 3;  // this lane finishes force component lane4
  const unsigned full = 0xffffffffu;
  const int a1 = lane4 & 1, a2 = lane4 >> 1;
  // every independent load first: positions, the lane's particle data, the
  // dipole accumulator and the step counter
  // use_mv: the move just made recorded the cell and sub-cell step of every
  // axis (the quantisation of the new position), so they are read instead of
  // computed again
  double xd = 0.0, vd = 0.0, gm = 0.0, sig = 0.0, hh = 0.0;
  int qi = 0, cq = 0, fq = 0;
  if (active) qi = P.q[p];
  if (comp) {
    // the move and its half kick may have been made in this launch by another
    // CTA (single-launch batch step): read through L2
    if (use_mv) {
      cq = __ldcg(P.mv + kMoveInts * p + 3 + lane4);
      fq = __ldcg(P.mv + kMoveInts * p + 6 + lane4);
    } else {
      xd = __ldcg(P.x + 3 * p + lane4);
    }
    vd = __ldcg(P.v + 3 * p + lane4);
    hh = P.h[p];
    if (thermo) {
      sig = P.sig[p];
      gm = P.gm[p];
    }
  }
  // pre (optional): the dipole sum and the step counter, read by the caller
  // (the warp's lanes all hold charges of one system: lane 0 reads it for the
  // warp, and lane 0 is active whenever any lane of its warp is)
  const int wlane = (threadIdx.x + blockDim.x * threadIdx.y) & 31;
  long long Pl[3] = {0, 0, 0};
  if (active && wlane == 0 && sp.dipole_corr) {
    Pl[0] = pre ? pre[0] : (long long)__ldcg(&ds->Pacc[0]);
    Pl[1] = pre ? pre[1] : (long long)__ldcg(&ds->Pacc[1]);
    Pl[2] = pre ? pre[2] : (long long)__ldcg(&ds->Pacc[2]);
  }
  unsigned rnd = 0;
  if (comp && thermo) {
    const long long step = pre ? pre[3] : __ldcg(&ds->step);
    unsigned ctr[4] = {(unsigned)p, (unsigned)((unsigned long long)p >> 32), (unsigned)step,
                       (unsigned)((unsigned long long)step >> 32)};
    philox4x32_10(ctr, (unsigned)sp.seed, (unsigned)(sp.seed >> 32));
    rnd = lane4 == 0 ? ctr[0] : (lane4 == 1 ? ctr[1] : ctr[2]);
  }
  // lane d < 3 quantises axis d; the quad shares the cells and sub-cell steps
  if (comp && !use_mv) quantize(m, lane4, xd, cq, fq);
  const int base = (threadIdx.x + blockDim.x * threadIdx.y) & 28;
  int c[3], f[3];
#pragma unroll
  for (int e = 0; e < 3; ++e) {
    c[e] = __shfl_sync(full, cq, base + e);
    f[e] = __shfl_sync(full, fq, base + e);
  }
  T E[3] = {T(0), T(0), T(0)};
  // 1/eps of the self term, summed in the field precision: the FP64 table
  // with FP64 fields, the field's own 1/eps with FP32 fields
  T iw[3] = {T(0), T(0), T(0)}, itot = T(0);
  if (active) {
    T Dv[3], Iv[3];
    double I64[3] = {0.0, 0.0, 0.0};
#pragma unroll
    for (int d = 0; d < 3; ++d) {
      const int e1 = (d + 1) % 3, e2 = (d + 2) % 3;
      int at[3] = {c[0], c[1], c[2]};
      at[e1] += a1;
      at[e2] += a2;
      const int64_t vtx = link_vertex(m, at[0], at[1], at[2]);
      const int64_t l = (int64_t)d * m.V + vtx;
      Dv[d] = __ldcg(D + l);  // D was updated in this launch by other CTAs (single launch)
      Iv[d] = ie[l];
      if (sp.self_mode != 0 && sizeof(T) == 8) I64[d] = ie64[l];
      if (Tpend) {  // transfers of this step not yet applied: as their application rounds
        const long long t = __ldcg(Tpend + tw_index(d, vtx, m.V));  // the step's own buffer
        if (t != 0) Dv[d] = Dv[d] + pending_inc<T>(t, sp.scale, exact32);
      }
    }
#pragma unroll
    for (int d = 0; d < 3; ++d) {
      const int e1 = (d + 1) % 3, e2 = (d + 2) % 3;
      const T w = ((T)wgt(f[e1], a1) / (T)kS) * ((T)wgt(f[e2], a2) / (T)kS);
      E[d] = Dv[d] * Iv[d] * w;
      const T iv = sizeof(T) == 8 ? (T)I64[d] : Iv[d];
      if (sp.self_mode != 0) itot += iv;
      if (sp.self_mode == 2) {
        const T wd = ((T)wgt(f[e1], a1) / (T)kS) * ((T)wgt(f[e2], a2) / (T)kS);
        iw[d] = iv * wd;
      }
    }
  }
  // quad sums in corner order ((c0 + c1) + (c2 + c3))
#pragma unroll
  for (int d = 0; d < 3; ++d) {
    E[d] = E[d] + __shfl_xor_sync(full, E[d], 1);
    E[d] = E[d] + __shfl_xor_sync(full, E[d], 2);
  }
  if (sp.self_mode == 2) {
#pragma unroll
    for (int d = 0; d < 3; ++d) {
      iw[d] = iw[d] + __shfl_xor_sync(full, iw[d], 1);
      iw[d] = iw[d] + __shfl_xor_sync(full, iw[d], 2);
    }
  }
  if (sp.self_mode != 0) {
    itot = itot + __shfl_xor_sync(full, itot, 1);
    itot = itot + __shfl_xor_sync(full, itot, 2);
  }
  // dipole force per unit charge, M P per component, computed by lane 0 for
  // the warp (same expression and rounding for every lane) and broadcast
  T MPw[3] = {T(0), T(0), T(0)};
  if (sp.dipole_corr) {
    if (wlane == 0)
#pragma unroll
      for (int e = 0; e < 3; ++e)
        MPw[e] = sp_Mdip<T>(sp, 3 * e) * (T)Pl[0] + sp_Mdip<T>(sp, 3 * e + 1) * (T)Pl[1] +
                 sp_Mdip<T>(sp, 3 * e + 2) * (T)Pl[2];
#pragma unroll
    for (int e = 0; e < 3; ++e) MPw[e] = __shfl_sync(full, MPw[e], 0);
  }
  if (comp) {
    // field force terms (q E, self energy, dipole) in R = T: FP64 with FP64
    // fields, FP32 with FP32 fields; the Langevin force, the velocity and the
    // kick stay FP64 (a single-precision noise of amplitude sqrt(2 gamma m
    // kT / dt) would move the velocities by more than the field rounding)
    using R = T;
    const int d = lane4;
    const R q = (R)qi;
    const T Ed = d == 0 ? E[0] : (d == 1 ? E[1] : E[2]);
    R F = q * (R)Ed;
    if (sp.self_mode != 0) {
      const R ie_cell = (R)itot * (R(1) / R(12));
      const R iwd = d == 0 ? iw[0] : (d == 1 ? iw[1] : iw[2]);
      const R ie_d = (sp.self_mode == 2) ? iwd : ie_cell;
      const SelfC<R> sc = self_coeffs<R>(f);
      F = F + (q * q * sp_self_pre<R>(sp)) * ie_d * self_sum<R>(sp, sc, d);
    }
    if (sp.dipole_corr) {
      const R MP = d == 0 ? MPw[0] : (d == 1 ? MPw[1] : MPw[2]);
      F = F + q * MP;
    }
    const double Fd = (double)F;
    double Ft = Fd;
    if (thermo) {
      const double fr = gm * vd;  // (-gamma m) v
      const double fn = sig * unit_noise(rnd);
      Ft = Fd + (fr + fn);
    }
    P.F[3 * p + d] = Fd;
    P.Ft[3 * p + d] = Ft;
    if (kick) P.v[3 * p + d] = __dadd_rn(vd, __dmul_rn(hh, Ft));
  }
  if (finish) finish_update(ds, finish, nctas);
}

template <typename T>
__global__ void __launch_bounds__(kQuadThreads)
    k_gather(const __grid_constant__ Mesh m, const __grid_constant__ StepParams sp, Particles P, const T* __restrict__ D, const T* __restrict__ ie,
             const double* __restrict__ ie64, DevState* ds, int kick, int finish) {
  // kick: the step's gather, right after the move that recorded the cells
  gather_body<T>(m, sp, sp.thermo, sp.gamma, sp.kT, P, D, ie, ie64, ds, kick, finish, gridDim.x,
                 blockIdx.x * (int64_t)blockDim.x + threadIdx.x, nullptr, false, nullptr,
                 kick != 0);
}

// One thread per charge: the gather of gather_body with the same
// expressions and the same order of every sum (each corner's three links,
// then the corners as ((c0 + c1) + (c2 + c3))), one Philox block a charge.
template <typename T>
__device__ __forceinline__ void gather_wide(const Mesh& m, const StepParams& sp, int thermo,
                                            Particles P, const T* __restrict__ D,
                                            const T* __restrict__ ie,
                                            const double* __restrict__ ie64, DevState* ds,
                                            int kick, int64_t p, bool use_mv) {
  if (p >= P.n) return;
  const int qi = P.q[p];
  int c[3], f[3];
#pragma unroll
  for (int d = 0; d < 3; ++d) {
    if (use_mv) {
      c[d] = __ldcg(P.mv + kMoveInts * p + 3 + d);
      f[d] = __ldcg(P.mv + kMoveInts * p + 6 + d);
    } else {
      quantize(m, d, __ldcg(P.x + 3 * p + d), c[d], f[d]);
    }
  }
  long long Pl[3] = {0, 0, 0};
  if (sp.dipole_corr) {
    Pl[0] = (long long)__ldcg(&ds->Pacc[0]);
    Pl[1] = (long long)__ldcg(&ds->Pacc[1]);
    Pl[2] = (long long)__ldcg(&ds->Pacc[2]);
  }
  unsigned ctr[4] = {0u, 0u, 0u, 0u};
  if (thermo) {
    const long long step = __ldcg(&ds->step);
    ctr[0] = (unsigned)p;
    ctr[1] = (unsigned)((unsigned long long)p >> 32);
    ctr[2] = (unsigned)step;
    ctr[3] = (unsigned)((unsigned long long)step >> 32);
    philox4x32_10(ctr, (unsigned)sp.seed, (unsigned)(sp.seed >> 32));
  }
  T Ek[4][3], iwk[4][3], itk[4];
#pragma unroll
  for (int k = 0; k < 4; ++k) {
    const int a1 = k & 1, a2 = k >> 1;
    T Dv[3], Iv[3];
    double I64[3] = {0.0, 0.0, 0.0};
#pragma unroll
    for (int d = 0; d < 3; ++d) {
      const int e1 = (d + 1) % 3, e2 = (d + 2) % 3;
      int at[3] = {c[0], c[1], c[2]};
      at[e1] += a1;
      at[e2] += a2;
      const int64_t l = link_index(m, d, at[0], at[1], at[2]);
      Dv[d] = __ldcg(D + l);
      Iv[d] = ie[l];
      if (sp.self_mode != 0 && sizeof(T) == 8) I64[d] = ie64[l];
    }
    itk[k] = T(0);
#pragma unroll
    for (int d = 0; d < 3; ++d) {
      const int e1 = (d + 1) % 3, e2 = (d + 2) % 3;
      const T w = ((T)wgt(f[e1], a1) / (T)kS) * ((T)wgt(f[e2], a2) / (T)kS);
      Ek[k][d] = Dv[d] * Iv[d] * w;
      const T iv = sizeof(T) == 8 ? (T)I64[d] : Iv[d];
      itk[k] += iv;
      iwk[k][d] = iv * w;
    }
  }
  using R = T;
  const R q = (R)qi;
  const R itot = (itk[0] + itk[1]) + (itk[2] + itk[3]);
  const SelfC<R> sc = self_coeffs<R>(f);
  const double hh = P.h[p];
  double sig = 0.0, gm = 0.0;
  if (thermo) {
    sig = P.sig[p];
    gm = P.gm[p];
  }
#pragma unroll
  for (int d = 0; d < 3; ++d) {
    const T Ed = (Ek[0][d] + Ek[1][d]) + (Ek[2][d] + Ek[3][d]);
    R F = q * (R)Ed;
    if (sp.self_mode != 0) {
      const R ie_cell = (R)itot * (R(1) / R(12));
      const R iwd = (iwk[0][d] + iwk[1][d]) + (iwk[2][d] + iwk[3][d]);
      const R ie_d = (sp.self_mode == 2) ? iwd : ie_cell;
      F = F + (q * q * sp_self_pre<R>(sp)) * ie_d * self_sum<R>(sp, sc, d);
    }
    if (sp.dipole_corr) {
      const R MP = sp_Mdip<T>(sp, 3 * d) * (T)Pl[0] + sp_Mdip<T>(sp, 3 * d + 1) * (T)Pl[1] +
                   sp_Mdip<T>(sp, 3 * d + 2) * (T)Pl[2];
      F = F + q * MP;
    }
    const double vd = __ldcg(P.v + 3 * p + d);
    const double Fd = (double)F;
    double Ft = Fd;
    if (thermo) {
      const double fr = gm * vd;  // (-gamma m) v
      const double fn = sig * unit_noise(ctr[d]);
      Ft = Fd + (fr + fn);
    }
    P.F[3 * p + d] = Fd;
    P.Ft[3 * p + d] = Ft;
    if (kick) P.v[3 * p + d] = __dadd_rn(vd, __dmul_rn(hh, Ft));
  }
}

template <typename T>
__global__ void __launch_bounds__(kWideThreads)
    k_gather_wide(const __grid_constant__ Mesh m, const __grid_constant__ StepParams sp,
                  Particles P, const T* __restrict__ D, const T* __restrict__ ie,
                  const double* __restrict__ ie64, DevState* ds, int kick, int finish) {
  gather_wide<T>(m, sp, sp.thermo, P, D, ie, ie64, ds, kick,
                 blockIdx.x * (int64_t)blockDim.x + threadIdx.x, kick != 0);
  if (finish) finish_update(ds, finish, gridDim.x);
}

// ------------------------------------------------------- batched replicas
// CTA b works on particles of replica cta_rep[b]; a replica's CTAs form a
// contiguous range, so warps and CTAs never mix replicas.
__device__ inline int64_t batch_local(const RepDesc& r) {
  return (int64_t)(blockIdx.x - r.p_first) * blockDim.x + threadIdx.x;
}

__global__ void __launch_bounds__(kBatchQuadThreads)
    k_deposit_batch(const RepDesc* __restrict__ desc, const int* __restrict__ cta_rep, int thermo,
                    double gamma, double kT) {
  const RepDesc& r = desc[cta_rep[blockIdx.x]];
  cta_dipole_add(r.ds->Pacc,
                 deposit_body(r.m, r.sp, r.P, (unsigned long long*)r.Tb, r.ds, batch_local(r)));
}

template <typename T>
__global__ void __launch_bounds__(kBatchQuadThreads)
    k_apply_batch(const RepDesc* __restrict__ desc, const int* __restrict__ cta_rep, int par) {
  const RepDesc& r = desc[cta_rep[blockIdx.x]];
  apply_body<T>(r.m, r.P, (unsigned long long*)r.Tb, r.Lg, (T*)r.D[par ^ 1], r.sp.scale,
                batch_local(r));
}

template <typename T>
__global__ void __launch_bounds__(kApplyThreads)
    k_apply_dense_batch(const RepDesc* __restrict__ desc, const int2* __restrict__ chunk,
                        int par) {
  const int2 c = chunk[blockIdx.x];
  const RepDesc& r = desc[c.x];
  const int64_t nl = 3 * r.m.V, l0 = (int64_t)c.y * kApplyChunk;
  apply_dense_range<T>(r.Tb, r.Lg, (T*)r.D[par ^ 1], r.sp.scale, l0,
                       l0 + kApplyChunk < nl ? l0 + kApplyChunk : nl, r.m.V);
}

template <typename T>
__global__ void __launch_bounds__(kBatchQuadThreads)
    k_gather_batch(const RepDesc* __restrict__ desc, const int* __restrict__ cta_rep, int par,
                   int thermo, double gamma, double kT) {
  const RepDesc& r = desc[cta_rep[blockIdx.x]];
  gather_body<T>(r.m, r.sp, thermo, gamma, kT, r.P, (const T*)r.D[par ^ 1], (const T*)r.ie, r.ie64, r.ds, 1, 2,
                 (unsigned)r.p_ctas, batch_local(r), nullptr, false, nullptr, true);
}

// one thread per charge: CTA b works on charges of replica cta_rep_w[b]
__device__ inline int64_t batch_local_w(const RepDesc& r) {
  return (int64_t)(blockIdx.x - r.pw_first) * blockDim.x + threadIdx.x;
}

// Seven CTAs an SM (at most 72 registers, a few words spilled to L1) hold
// a 64-replica batch's ~1000 CTAs in one wave; at the 88 registers the
// kernel takes unbounded, five fit and a second wave trails (42.4 -> 38.5 us
// a launch on 124k charges).
__global__ void __launch_bounds__(kWideThreads, 7)
    k_deposit_batch_wide(const RepDesc* __restrict__ desc, const int* __restrict__ cta_rep) {
  const RepDesc& r = desc[cta_rep[blockIdx.x]];
  long long U[3];
  deposit_wide(r.m, r.sp, r.P, (unsigned long long*)r.Tb, r.ds, batch_local_w(r), U);
  cta_dipole_add3(r.ds->Pacc, U);
}

template <typename T>
__global__ void __launch_bounds__(kWideThreads)
    k_gather_batch_wide(const RepDesc* __restrict__ desc, const int* __restrict__ cta_rep,
                        int par, int thermo) {
  const RepDesc& r = desc[cta_rep[blockIdx.x]];
  gather_wide<T>(r.m, r.sp, thermo, r.P, (const T*)r.D[par ^ 1], (const T*)r.ie, r.ie64, r.ds, 1,
                 batch_local_w(r), true);
  finish_update(r.ds, 2, (unsigned)r.pw_ctas);
}

// ------------------------------------------- single-launch batch step
__device__ inline unsigned long long ld_acquire_u64(const unsigned long long* p) {
  unsigned long long v;
  asm volatile("ld.acquire.gpu.global.u64 %0, [%1];" : "=l"(v) : "l"(p) : "memory");
  return v;
}
__device__ inline unsigned long long ld_relaxed_u64(const unsigned long long* p) {
  unsigned long long v;
  asm volatile("ld.relaxed.gpu.global.u64 %0, [%1];" : "=l"(v) : "l"(p) : "memory");
  return v;
}
__device__ inline unsigned long long add_acq_rel_u64(unsigned long long* p, unsigned long long v) {
  unsigned long long r;
  asm volatile("atom.acq_rel.gpu.global.add.u64 %0, [%1], %2;" : "=l"(r) : "l"(p), "l"(v) : "memory");
  return r;
}
__device__ inline unsigned long long global_ns() {
  unsigned long long t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}

// Warp 0 of a CTA claims its next item.  Dependent work first: lane l looks
// at replica cursor + l (32 at a time); a replica's gather items are
// claimable when all its application items have finished, its application
// items when all its field segments and deposition items have, and some of
// them are not yet claimed; the lowest such replica (gathers before
// applications: they finish replicas) is claimed with one atomic add on its
// own count (a count past the end means another CTA took the last item: look
// again).  Then independent work: field segments first for field CTAs,
// deposition items first for the others.  A CTA waits only when every
// independent item has been claimed and no dependent item is ready; dependent
// items are claimed only when ready and so never wait once claimed, and the
// ones left depend only on claimed items, so the wait ends.  It is bounded by
// the global timer all the same (kErrTimeout, and the CTA leaves).  Returns
// the kind (setting *rep and *item) or -1 when nothing is left; every lane of
// warp 0 gets the same answer.
__device__ int batch_claim(const BatchStepArgs& a, unsigned long long e1, bool field_first,
                           bool& fdone, bool& ddone, int& cursor, int* rep, int* item) {
  const unsigned full = 0xffffffffu;
  const int lane = threadIdx.x & 31;
  BatchSched* S = a.sched;
  unsigned long long t0 = 0;
  for (;;) {
    bool left = false;  // some replica has dependent items not yet claimed
    for (int r0 = cursor; r0 < a.nrep; r0 += 32) {
      const int r = r0 + lane;
      bool cg = false, ca = false, gone = true;
      unsigned long long np = 0;
      if (r < a.nrep) {
        const RepDesc& d = a.desc[r];
        RepSync& y = a.sync[r];
        np = (unsigned long long)d.b_np;
        const unsigned long long ka = ld_relaxed_u64(&y.claim[0]) - y.base[0];
        const unsigned long long kg = ld_relaxed_u64(&y.claim[1]) - y.base[1];
        gone = ka >= np && kg >= np;
        if (kg < np) cg = ld_acquire_u64(&y.done[kItemApply]) >= e1 * np;
        if (!cg && ka < np)
          ca = ld_acquire_u64(&y.done[kItemField]) >= e1 * (unsigned long long)d.b_nf &&
               ld_acquire_u64(&y.done[kItemDeposit]) >= e1 * np;
      }
      const unsigned bg = __ballot_sync(full, cg), ba = __ballot_sync(full, ca);
      const unsigned bgone = __ballot_sync(full, gone);
      if (r0 == cursor) cursor += bgone == full ? 32 : __ffs(~bgone) - 1;  // skip finished
      left = left || bgone != full;
      if (bg | ba) {
        const int src = bg ? __ffs(bg) - 1 : __ffs(ba) - 1;
        const int kind = bg ? kItemGather : kItemApply;
        unsigned long long k = 0;
        if (lane == src) k = atomicAdd(&a.sync[r].claim[kind - kItemApply], 1ull) - a.sync[r].base[kind - kItemApply];
        k = __shfl_sync(full, k, src);
        const unsigned long long nps = __shfl_sync(full, np, src);
        if (k < nps) {
          *rep = r0 + src;
          *item = (int)k;
          return kind;
        }
        r0 -= 32;  // another CTA took the last one: look at these replicas again
        continue;
      }
    }
    int q = -1, k = 0;
    if (lane == 0) {
      const int first = field_first ? kItemField : kItemDeposit;
      for (int j = 0; j < 2 && q < 0; ++j) {
        const int qq = j == 0 ? first : kItemField + kItemDeposit - first;
        bool& done = qq == kItemField ? fdone : ddone;
        if (done) continue;
        const unsigned long long c = atomicAdd(&S->next[qq], 1ull) - S->base[qq];
        if (c < (unsigned long long)a.n[qq]) {
          q = qq;
          k = (int)c;
        } else {
          done = true;
        }
      }
    }
    q = __shfl_sync(full, q, 0);
    fdone = __shfl_sync(full, fdone, 0);
    ddone = __shfl_sync(full, ddone, 0);
    if (q >= 0) {
      k = __shfl_sync(full, k, 0);
      *rep = a.q[q][k].rep;
      *item = k;
      return q;
    }
    if (!left) return -1;
    unsigned long long t = 0;
    if (lane == 0) t = global_ns();
    t = __shfl_sync(full, t, 0);
    if (t0 == 0) {
      t0 = t;
    } else if (t - t0 > a.wait_ns) {
      if (lane == 0) atomicOr(&S->err, kErrTimeout);
      return -1;
    }
    __nanosleep(200);
  }
}

// The step of every replica in one cooperative launch (see BatchStepArgs).
// Each item runs on the whole CTA; its completion is published by thread 0
// after the CTA's barrier (a gpu-scope fence, then an acquire-release count).
// The CTA that completes a replica's last gather item closes that replica's
// step (P of this state reported, the sum cleared, the counter advanced), and
// the last CTA to leave moves the claim bases and the launch count on.
template <typename T>
__global__ void __launch_bounds__(kBatchStepThreads, 2)
    k_batch_step(const __grid_constant__ BatchStepArgs a) {
  extern __shared__ __align__(16) unsigned char bs_smem[];
  __shared__ int s_kind, s_rep, s_item, s_last;
  BatchSched* S = a.sched;
  const unsigned long long e1 = ld_relaxed_u64(&S->epoch) + 1;
  bool fdone = false, ddone = false;
  int cursor = 0;
  const bool field_first = (int)blockIdx.x < a.field_ctas;
  for (;;) {
    if (threadIdx.x < 32) {
      int rep = 0, item = 0;
      const int kind = batch_claim(a, e1, field_first, fdone, ddone, cursor, &rep, &item);
      if (threadIdx.x == 0) {
        s_kind = kind;
        s_rep = rep;
        s_item = item;
      }
    }
    __syncthreads();
    const int kind = s_kind;
    if (kind < 0) break;
    const int rep = s_rep, item = s_item;
    const RepDesc& r = a.desc[rep];
    if (kind == kItemField) {
      const BatchItem it = a.q[kItemField][item];
      unsigned char* stg = bs_smem;
      T* sE = reinterpret_cast<T*>(bs_smem + (size_t)3 * 6 * kBatchStepThreads * 16);
      T* sB = sE + 3 * (it.b + 2) * r.m.n[0];
      rows::rows_segment<T, kBatchStepThreads>(
          r.m, (const T*)r.D[a.par], (const T*)r.B[a.par], (const T*)r.ie, (T*)r.D[a.par ^ 1],
          (T*)r.B[a.par ^ 1], (T)r.sp.coefB, (T)r.sp.coefD, it.a, it.b, it.c, it.d, sE, sB, stg);
    } else {
      // the item's chunks of kBatchStepThreads quad lanes
      const int k = kind == kItemDeposit ? a.q[kItemDeposit][item].a : item;
      const int c1 = min((k + 1) * kBatchChunksPerItem, r.b_nc);
      for (int c = k * kBatchChunksPerItem; c < c1; ++c) {
        const int64_t g = (int64_t)c * kBatchStepThreads + threadIdx.x;
        if (kind == kItemDeposit)
          cta_dipole_add(r.ds->Pacc,
                         deposit_body(r.m, r.sp, r.P, (unsigned long long*)r.Tb, r.ds, g));
        else if (kind == kItemApply)
          apply_body<T>(r.m, r.P, (unsigned long long*)r.Tb, r.Lg, (T*)r.D[a.par ^ 1],
                        r.sp.scale, g);
        else
          gather_body<T>(r.m, r.sp, a.thermo, a.gamma, a.kT, r.P, (const T*)r.D[a.par ^ 1],
                         (const T*)r.ie, r.ie64, r.ds, 1, 0, 0, g, nullptr, false, nullptr, true);
      }
    }
    __syncthreads();  // the item is done (and s_kind, s_rep, s_item read by every thread)
    if (threadIdx.x == 0) {
      __threadfence();
      const unsigned long long t = add_acq_rel_u64(&a.sync[rep].done[kind], 1ull);
      if (kind == kItemGather && t + 1 == e1 * (unsigned long long)r.b_np) {
        DevState* ds = r.ds;
        const unsigned long long p0 = __ldcg(&ds->Pacc[0]), p1 = __ldcg(&ds->Pacc[1]),
                                 p2 = __ldcg(&ds->Pacc[2]);
        ds->Plast[0] = (long long)p0;
        ds->Plast[1] = (long long)p1;
        ds->Plast[2] = (long long)p2;
        ds->Pacc[0] = 0ull;
        ds->Pacc[1] = 0ull;
        ds->Pacc[2] = 0ull;
        ds->step = __ldcg(&ds->step) + 1;
      }
    }
  }
  if (threadIdx.x == 0) {
    const unsigned long long t = add_acq_rel_u64(&S->exits, 1ull);
    s_last = (t + 1) % gridDim.x == 0;
  }
  __syncthreads();
  if (s_last) {
    // every CTA has left: all claims of this launch are made
    __threadfence();
    for (int r = threadIdx.x; r < a.nrep; r += blockDim.x) {
      RepSync& y = a.sync[r];
      y.base[0] = ld_relaxed_u64(&y.claim[0]);
      y.base[1] = ld_relaxed_u64(&y.claim[1]);
    }
    if (threadIdx.x == 0) {
      S->base[0] = ld_relaxed_u64(&S->next[0]);
      S->base[1] = ld_relaxed_u64(&S->next[1]);
      S->epoch = e1;
    }
  }
}

// ---------------------------------------------------- single-launch step
// The whole time step of one system in one cooperative launch of G CTAs,
// with one grid barrier.  The transfers of a step are applied lazily: they
// stay in the transfer buffer Tcur, the gather reads D + Tcur scale (rounded
// as their application rounds), and the next step's field tiles read their
// D the same way from that buffer (then Tprev) before updating it; after
// that step's barrier the field warps move Tprev into the ledger and clear
// it.  Phase 1: warps 0-10 of every CTA run field tiles (B' then D',
// one-thread-per-site tiles of 8 rows) while warp 11 runs the kick, drift
// and deposition into Tcur; grid barrier; phase 2: warp 11 gathers the
// forces (Langevin, half kick) while the field warps commit Tprev; the last
// CTA closes the step.  The values are those of the four launches of the
// graph step, bit for bit.

// Grid-wide barrier of a cooperative launch over a monotonic 64-bit count
// of CTA arrivals: each CTA adds one with release and acquire semantics and
// learns its arrival number a; its barrier is complete when the count
// reaches the next multiple of the grid size (the count starts at 0 and
// grows by exactly the grid size a barrier).  The last CTA to arrive knows
// it from a alone and goes on; the others poll the count with relaxed loads
// and acquire once it is reached.  The arrivals are read-modify-writes of one
// word, so they form one release sequence: the last arrival, and a poll that
// reads the completed count, acquire every CTA's earlier writes.  The wait is bounded
// by the global timer (0.2 s); a wait that runs out sets kErrTimeout and
// goes on, the step is then void and the host resets the count when it
// reports the error.
__device__ inline void grid_barrier(DevState* ds, unsigned nctas, unsigned long long wait_ns) {
  __syncthreads();
  if (threadIdx.x == 0) {
    unsigned long long a;
    asm volatile("atom.acq_rel.gpu.global.add.u64 %0, [%1], 1;"
                 : "=l"(a)
                 : "l"(&ds->bar_arrivals)
                 : "memory");
    const unsigned long long target = a - a % nctas + nctas;
    if (a + 1 != target) {
      unsigned long long t0, t, cur;
      asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t0));
      for (unsigned it = 1;; ++it) {
        asm volatile("ld.relaxed.gpu.global.u64 %0, [%1];"
                     : "=l"(cur)
                     : "l"(&ds->bar_arrivals)
                     : "memory");
        if (cur >= target) break;
        if ((it & 255u) == 0u) {
          asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
          if (t - t0 > wait_ns) {
            atomicOr(&ds->err, kErrTimeout);
            break;
          }
        }
      }
      asm volatile("fence.acq_rel.gpu;" ::: "memory");
    }
  }
  __syncthreads();
}

// barrier of the field warps of a CTA (named barrier 1)
struct FieldWarpsSync {
  __device__ void operator()() const {
    asm volatile("barrier.sync.aligned 1, %0;" ::"n"(32 * kCoopFieldWarps) : "memory");
  }
};

// ledger += Tprev, Tprev = 0 on the sites a field thread updates
__device__ __forceinline__ void commit_tile(const Mesh& m, int txi, int tyi, int tz, int zchunk,
                                            int tx, int ty, bool live, long long* __restrict__ Tp,
                                            long long* __restrict__ Lg) {
  const int nx = m.n[0], ny = m.n[1];
  const int x = txi * 32 - 1 + tx, y = tyi * 8 - 1 + ty;
  if (!live || tx < 1 || tx > 32 || ty < 1 || ty > 8 || x >= nx || y >= ny) return;
  const int z0 = tz * zchunk, z1 = min(z0 + zchunk, m.n[2]);
  const int64_t P = (int64_t)nx * ny;
  for (int k = z0; k < z1; ++k)
#pragma unroll
    for (int c = 0; c < 3; ++c) {
      const int64_t v = (int64_t)k * P + (int64_t)y * nx + x;
      const int64_t w = tw_index(c, v, m.V);  // the step's own buffer: component major
      const long long t = Tp[w];
      if (t != 0) {
        Lg[kLT * tl_pair(c, v)] += t;
        Tp[w] = 0;
      }
    }
}

template <typename T>
__global__ void __launch_bounds__(kCoopThreads)
    k_step_coop(const __grid_constant__ Mesh m, const __grid_constant__ StepParams sp, Particles P,
                const T* __restrict__ Din, const T* __restrict__ Bin, const T* __restrict__ ie,
                T* __restrict__ Dout, T* __restrict__ Bout, const double* __restrict__ ie64,
                long long* __restrict__ Tprev, unsigned long long* __restrict__ Tcur,
                long long* __restrict__ Lg, DevState* ds, int zchunk) {
  const bool exact32 = m.a_pow2 != 0;  // power-of-two scale (FP32 fields use it)
  const int tid = threadIdx.x;
  const bool pwarp = (tid >> 5) == kCoopFieldWarps;
  const unsigned G = gridDim.x;
  const int lane = tid & 31;
  const int64_t nq = 4 * P.n;  // quad lanes of all particles
  const int64_t stride = (int64_t)G * 32;
  const int tiles_x = (m.n[0] + 31) / 32, tiles_y = (m.n[1] + 7) / 8;
  const int tiles_z = (m.n[2] + zchunk - 1) / zchunk;
  const int ntiles = tiles_x * tiles_y * tiles_z;
  const bool live = tid < 34 * 10;
  const int tx = live ? tid % 34 : 0, ty = live ? tid / 34 : 0;
  if (!pwarp) {
    for (int t = blockIdx.x; t < ntiles; t += (int)G) {
      const int tz = t / (tiles_x * tiles_y), r = t - tz * (tiles_x * tiles_y);
      const int tyi = r / tiles_x, txi = r - tyi * tiles_x;
      site_tile<T, 8, 1>(m, Din, Bin, ie, Dout, Bout, (T)sp.coefB, (T)sp.coefD, txi, tyi, tz,
                         zchunk, tx, ty, live, FieldWarpsSync{}, Tprev, sp.scale, exact32);
    }
  } else {
    for (int64_t b = (int64_t)blockIdx.x * 32; b < nq; b += stride)
      quad_dipole_add(ds->Pacc, deposit_body(m, sp, P, Tcur, ds, b + lane, (const char*)ie,
                                             (int)sizeof(T), m.V));
  }
  grid_barrier(ds, G, sp.wait_ns);
  if (pwarp) {
    // the dipole sum of this move and the step counter, read once; the
    // particle warp then signals field warp 0 (named barrier 2), which takes
    // the CTA's ticket while the gather runs, so the last CTA closes the step
    // (P of this state reported, the sum cleared, the counter advanced) off
    // the gather's path.  Every CTA's reads are complete before its signal:
    // the signal consumes them.
    long long pre[4];
    pre[0] = (long long)__ldcg(&ds->Pacc[0]);
    pre[1] = (long long)__ldcg(&ds->Pacc[1]);
    pre[2] = (long long)__ldcg(&ds->Pacc[2]);
    pre[3] = __ldcg(&ds->step);
    const long long used = ((pre[0] ^ pre[1]) ^ pre[2]) ^ pre[3];
    asm volatile("bar.arrive 2, 64;" ::"l"(used) : "memory");
    for (int64_t b = (int64_t)blockIdx.x * 32; b < nq; b += stride)
      gather_body<T>(m, sp, sp.thermo, sp.gamma, sp.kT, P, Dout, ie, ie64, ds, 1, 0, G, b + lane,
                     (const long long*)Tcur, exact32, pre, true);
  } else {
    for (int t = blockIdx.x; t < ntiles; t += (int)G) {
      const int tz = t / (tiles_x * tiles_y), r = t - tz * (tiles_x * tiles_y);
      const int tyi = r / tiles_x, txi = r - tyi * tiles_x;
      commit_tile(m, txi, tyi, tz, zchunk, tx, ty, live, Tprev, Lg);
    }
    if (tid < 32) {
      asm volatile("bar.sync 2, 64;" ::: "memory");
      if (tid == 0) {
        unsigned t;
        asm volatile("atom.acq_rel.gpu.global.add.u32 %0, [%1], 1;"
                     : "=r"(t)
                     : "l"(&ds->ticket)
                     : "memory");
        if (t == G - 1) {
          const unsigned long long p0 = __ldcg(&ds->Pacc[0]), p1 = __ldcg(&ds->Pacc[1]),
                                   p2 = __ldcg(&ds->Pacc[2]);
          const long long st = __ldcg(&ds->step);
          ds->Plast[0] = (long long)p0;
          ds->Plast[1] = (long long)p1;
          ds->Plast[2] = (long long)p2;
          ds->Pacc[0] = 0ull;
          ds->Pacc[1] = 0ull;
          ds->Pacc[2] = 0ull;
          ds->step = st + 1;
          ds->ticket = 0u;
        }
      }
    }
  }
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
      double ie_cell, ie_dir[3];
      self_ie(m, ie64, c, f, sp.self_mode, ie_cell, ie_dir);
      const SelfC<double> sc = self_coeffs<double>(f);
      const double q = (double)P.q[p];
      se += q * q / (2.0 * m.a) * ie_cell * self_sum<double>(sp, sc, -1);
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

// One block of host I/O (memd_step_io): positions, velocities (n x 3
// doubles each), image counters (n x 3 ints, padded to 8 bytes), forces
// (n x 3 doubles), the error word.  unpack loads a state from it (positions
// folded as at init), pack writes the state and forces back into it.
// particle p of a system from block entry e (the same index for a single
// system; the system's offset plus p in a batch block)
__device__ inline void io_unpack_one(const Mesh& m, Particles P, const IoLayout& L,
                                     const unsigned char* __restrict__ io, int64_t p, int64_t e,
                                     unsigned int* err) {
  const double* pos = reinterpret_cast<const double*>(io + L.pos);
  const double* vel = reinterpret_cast<const double*>(io + L.vel);
  const int* img = reinterpret_cast<const int*>(io + L.img);
  for (int d = 0; d < 3; ++d) {
    double x = pos[3 * e + d];
    int k = img[3 * e + d];
    if (!(fabs(x) <= 4.0 * m.L[d])) {
      atomicOr(err, kErrNonFinite);
      x = 0.0;
    }
    fold(m.L[d], x, k);
    P.x[3 * p + d] = x;
    P.img[3 * p + d] = k;
    P.v[3 * p + d] = vel[3 * e + d];
  }
}

__device__ inline void io_pack_one(Particles P, const IoLayout& L, unsigned char* __restrict__ io,
                                   int64_t p, int64_t e, int part = kIoAll) {
  double* pos = reinterpret_cast<double*>(io + L.pos);
  double* vel = reinterpret_cast<double*>(io + L.vel);
  int* img = reinterpret_cast<int*>(io + L.img);
  double* f = reinterpret_cast<double*>(io + L.f);
  for (int d = 0; d < 3; ++d) {
    if (part != kIoRest) {
      pos[3 * e + d] = P.x[3 * p + d];
      img[3 * e + d] = P.img[3 * p + d];
    }
    if (part != kIoMoved) {
      vel[3 * e + d] = P.v[3 * p + d];
      f[3 * e + d] = P.F[3 * p + d];
    }
  }
}

__global__ void k_io_unpack(Mesh m, Particles P, const unsigned char* __restrict__ io,
                            unsigned int* err) {
  const int64_t p = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (p >= P.n) return;
  io_unpack_one(m, P, io_layout(P.n), io, p, p, err);
}

__global__ void k_io_pack(Particles P, unsigned char* __restrict__ io,
                          const unsigned int* __restrict__ err) {
  const int64_t p = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  const IoLayout L = io_layout(P.n);
  if (p == 0) *reinterpret_cast<unsigned int*>(io + L.err) = *err;
  if (p >= P.n) return;
  io_pack_one(P, L, io, p, p);
}

// The batch block: the members' particles one after another (member r from
// entry off[r]), laid out as one system of off[count] particles, the error
// words of the members after it.  Entry e belongs to the member r with
// off[r] <= e < off[r + 1] (binary search over count + 1 offsets).
__device__ inline int io_member(const int64_t* __restrict__ off, int count, int64_t e) {
  int lo = 0, hi = count;  // off[lo] <= e < off[hi]
  while (hi - lo > 1) {
    const int mid = (lo + hi) >> 1;
    if (off[mid] <= e)
      lo = mid;
    else
      hi = mid;
  }
  return lo;
}

__global__ void k_io_unpack_batch(const RepDesc* __restrict__ desc,
                                  const int64_t* __restrict__ off, int count,
                                  const unsigned char* __restrict__ io) {
  const int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  const int64_t ntot = off[count];
  if (e >= ntot) return;
  const int r = io_member(off, count, e);
  const RepDesc& d = desc[r];
  io_unpack_one(d.m, d.P, io_layout(ntot), io, e - off[r], e, &d.ds->err);
}

__global__ void k_io_pack_batch(const RepDesc* __restrict__ desc,
                                const int64_t* __restrict__ off, int count,
                                unsigned char* __restrict__ io, int part) {
  const int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  const int64_t ntot = off[count];
  const IoLayout L = io_layout(ntot);
  if (e < count && part != kIoMoved)
    reinterpret_cast<unsigned int*>(io + L.err)[e] = desc[e].ds->err;
  if (e >= ntot) return;
  const int r = io_member(off, count, e);
  io_pack_one(desc[r].P, L, io, e - off[r], e, part);
}

void launch_io_unpack(const Mesh& m, Particles p, const void* io, unsigned int* err,
                      cudaStream_t st) {
  if (p.n > 0)
    k_io_unpack<<<blocks_for(p.n), kThreads, 0, st>>>(m, p, (const unsigned char*)io, err);
}

void launch_io_pack(Particles p, void* io, const unsigned int* err, cudaStream_t st) {
  k_io_pack<<<blocks_for(p.n > 0 ? p.n : 1), kThreads, 0, st>>>(p, (unsigned char*)io, err);
}

void launch_io_unpack_batch(const RepDesc* desc, const int64_t* off, int count, int64_t ntot,
                            const void* io, cudaStream_t st) {
  if (ntot > 0)
    k_io_unpack_batch<<<blocks_for(ntot), kThreads, 0, st>>>(desc, off, count,
                                                            (const unsigned char*)io);
}

void launch_io_pack_batch(const RepDesc* desc, const int64_t* off, int count, int64_t ntot,
                          void* io, cudaStream_t st, int part) {
  k_io_pack_batch<<<blocks_for(ntot > count ? ntot : count), kThreads, 0, st>>>(
      desc, off, count, (unsigned char*)io, part);
}

void launch_fold_init(const Mesh& m, Particles p, const double* pos_in, const int* img_in,
                      unsigned int* err, cudaStream_t st) {
  if (p.n > 0) k_fold_init<<<blocks_for(p.n), kThreads, 0, st>>>(m, p, pos_in, img_in, err);
}

void launch_cic(const Mesh& m, Particles p, long long* Q, long long bg, cudaStream_t st) {
  cudaMemsetAsync(Q, 0, sizeof(long long) * m.V, st);
  if (p.n > 0) k_cic<<<blocks_for(p.n), kThreads, 0, st>>>(m, p, (unsigned long long*)Q);
  if (bg != 0) k_sub_background<<<blocks_for(m.V, 256), 256, 0, st>>>(m.V, Q, bg);
}

void launch_cic_abs(const Mesh& m, Particles p, long long* Q, cudaStream_t st) {
  cudaMemsetAsync(Q, 0, sizeof(long long) * m.V, st);
  if (p.n > 0) k_cic_abs<<<blocks_for(p.n), kThreads, 0, st>>>(m, p, (unsigned long long*)Q);
}

void launch_dipole(const Mesh& m, Particles p, DevState* ds, cudaStream_t st) {
  cudaMemsetAsync(ds->Pacc, 0, sizeof(ds->Pacc), st);
  if (p.n > 0) k_dipole<<<blocks_for(p.n), kThreads, 0, st>>>(m, p, ds);
}

void launch_particle_constants(const StepParams& sp, Particles p, cudaStream_t st) {
  if (p.n > 0) k_particle_constants<<<blocks_for(p.n), kThreads, 0, st>>>(sp, p);
}

void launch_kick_drift_deposit(const Mesh& m, const StepParams& sp, Particles p, long long* Tb,
                               DevState* ds, cudaStream_t st) {
  if (p.n >= kWideMinCharges)
    k_deposit_wide<<<blocks_for(p.n, kWideThreads), kWideThreads, 0, st>>>(
        m, sp, p, (unsigned long long*)Tb, ds);
  else if (p.n > 0)
    k_kick_drift_deposit<<<blocks_for(4 * p.n, quad_threads(p.n)), quad_threads(p.n), 0, st>>>(
        m, sp, p, (unsigned long long*)Tb, ds);
}

void launch_move_deposit(const Mesh& m, Particles p, const double* pos_new, const int* img_new,
                         long long* Tb, DevState* ds, cudaStream_t st) {
  if (p.n > 0)
    k_move_deposit<<<blocks_for(4 * p.n, quad_threads(p.n)), quad_threads(p.n), 0, st>>>(
        m, p, pos_new, img_new, (unsigned long long*)Tb, ds);
}

void launch_apply(const Mesh& m, int prec, Particles p, long long* Tb, long long* Lg, void* D,
                  double scale, cudaStream_t st, int64_t cmV) {
  if (p.n <= 0) return;
  const int qt = quad_threads(p.n);
  const unsigned nb = blocks_for(4 * p.n, qt);
  if (prec == 1)
    k_apply<float><<<nb, qt, 0, st>>>(m, p, (unsigned long long*)Tb, Lg, (float*)D, scale, cmV);
  else
    k_apply<double><<<nb, qt, 0, st>>>(m, p, (unsigned long long*)Tb, Lg, (double*)D, scale,
                                       cmV);
}

void launch_apply_dense(int prec, int64_t nlinks, long long* Tb, long long* Lg, void* D,
                        double scale, cudaStream_t st) {
  if (nlinks <= 0) return;
  const unsigned nb = (unsigned)((nlinks + kApplyChunk - 1) / kApplyChunk);
  if (prec == 1)
    k_apply_dense<float><<<nb, kApplyThreads, 0, st>>>(nlinks, Tb, Lg, (float*)D, scale);
  else
    k_apply_dense<double><<<nb, kApplyThreads, 0, st>>>(nlinks, Tb, Lg, (double*)D, scale);
}

size_t batch_step_smem() { return rows_smem_bytes(kBatchStepThreads, 4); }

namespace {
template <typename T>
cudaError_t batch_step_attr() {
  static cudaError_t done = cudaFuncSetAttribute(
      k_batch_step<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)batch_step_smem());
  return done;
}
}  // namespace

int batch_step_occupancy(int prec) {
  int n = 0;
  const cudaError_t e =
      prec == 1 ? (batch_step_attr<float>() != cudaSuccess
                       ? cudaErrorInvalidValue
                       : cudaOccupancyMaxActiveBlocksPerMultiprocessor(
                             &n, k_batch_step<float>, kBatchStepThreads, batch_step_smem()))
                : (batch_step_attr<double>() != cudaSuccess
                       ? cudaErrorInvalidValue
                       : cudaOccupancyMaxActiveBlocksPerMultiprocessor(
                             &n, k_batch_step<double>, kBatchStepThreads, batch_step_smem()));
  if (e != cudaSuccess) {
    cudaGetLastError();
    return 0;
  }
  return n;
}

cudaError_t launch_batch_step(int prec, const BatchStepArgs& a, int grid, cudaStream_t st) {
  cudaLaunchConfig_t cfg{};
  cfg.gridDim = dim3((unsigned)grid, 1, 1);
  cfg.blockDim = dim3(kBatchStepThreads, 1, 1);
  cfg.dynamicSmemBytes = batch_step_smem();
  cfg.stream = st;
  cudaLaunchAttribute at[1];
  at[0].id = cudaLaunchAttributeCooperative;
  at[0].val.cooperative = 1;
  cfg.attrs = at;
  cfg.numAttrs = 1;
  if (prec == 1) {
    const cudaError_t e = batch_step_attr<float>();
    return e != cudaSuccess ? e : cudaLaunchKernelEx(&cfg, k_batch_step<float>, a);
  }
  const cudaError_t e = batch_step_attr<double>();
  return e != cudaSuccess ? e : cudaLaunchKernelEx(&cfg, k_batch_step<double>, a);
}

int coop_grid(int prec, int device) {
  int coop = 0, sms = 0, per = 0;
  if (cudaDeviceGetAttribute(&coop, cudaDevAttrCooperativeLaunch, device) != cudaSuccess || !coop ||
      cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, device) != cudaSuccess) {
    cudaGetLastError();
    return 0;
  }
  const cudaError_t e =
      prec == 1 ? cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, k_step_coop<float>, kCoopThreads, 0)
                : cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, k_step_coop<double>, kCoopThreads, 0);
  if (e != cudaSuccess || per < 1) {
    cudaGetLastError();
    return 0;
  }
  return sms;  // one CTA per SM
}

int coop_zchunk(const Mesh& m, int grid) {
  const int tiles_xy = ((m.n[0] + 31) / 32) * ((m.n[1] + 7) / 8);
  int zc = 1;
  while (zc < m.n[2] && (int64_t)tiles_xy * ((m.n[2] + zc - 1) / zc) > grid) zc *= 2;
  return zc < m.n[2] ? zc : m.n[2];
}

cudaError_t launch_step_coop(const Mesh& m, int prec, const StepParams& sp, Particles p,
                             const void* Din, const void* Bin, const void* ie, void* Dout,
                             void* Bout, const double* ie64, long long* Tprev, long long* Tcur,
                             long long* Lg, DevState* ds, int grid, int zchunk, cudaStream_t st) {
  cudaLaunchConfig_t cfg{};
  cfg.gridDim = dim3((unsigned)grid, 1, 1);
  cfg.blockDim = dim3(kCoopThreads, 1, 1);
  cfg.dynamicSmemBytes = 0;
  cfg.stream = st;
  cudaLaunchAttribute at[1];
  at[0].id = cudaLaunchAttributeCooperative;
  at[0].val.cooperative = 1;
  cfg.attrs = at;
  cfg.numAttrs = 1;
  unsigned long long* tc = (unsigned long long*)Tcur;
  if (prec == 1)
    return cudaLaunchKernelEx(&cfg, k_step_coop<float>, m, sp, p, (const float*)Din,
                              (const float*)Bin, (const float*)ie, (float*)Dout, (float*)Bout, ie64,
                              Tprev, tc, Lg, ds, zchunk);
  return cudaLaunchKernelEx(&cfg, k_step_coop<double>, m, sp, p, (const double*)Din,
                            (const double*)Bin, (const double*)ie, (double*)Dout, (double*)Bout,
                            ie64, Tprev, tc, Lg, ds, zchunk);
}

void launch_gather(const Mesh& m, int prec, const StepParams& sp, Particles p, const void* D,
                   const void* ie, const double* ie64, DevState* ds, int kick, int finish,
                   cudaStream_t st) {
  if (p.n <= 0) {
    if (finish) k_step_end<<<1, 32, 0, st>>>(ds, finish == 2 ? 1 : 0);
    return;
  }
  if (p.n >= kWideMinCharges) {
    const unsigned nw = blocks_for(p.n, kWideThreads);
    if (prec == 1)
      k_gather_wide<float><<<nw, kWideThreads, 0, st>>>(m, sp, p, (const float*)D,
                                                        (const float*)ie, ie64, ds, kick, finish);
    else
      k_gather_wide<double><<<nw, kWideThreads, 0, st>>>(m, sp, p, (const double*)D,
                                                         (const double*)ie, ie64, ds, kick, finish);
    return;
  }
  const int qt = quad_threads(p.n);
  const unsigned nb = blocks_for(4 * p.n, qt);
  if (prec == 1)
    k_gather<float><<<nb, qt, 0, st>>>(m, sp, p, (const float*)D, (const float*)ie,
                                                 ie64, ds, kick, finish);
  else
    k_gather<double><<<nb, qt, 0, st>>>(m, sp, p, (const double*)D, (const double*)ie,
                                                  ie64, ds, kick, finish);
}

void launch_step_end(DevState* ds, int advance, cudaStream_t st) {
  k_step_end<<<1, 32, 0, st>>>(ds, advance);
}

void launch_deposit_batch(const RepDesc* desc, const int* cta_rep, int nctas, int thermo,
                          double gamma, double kT, cudaStream_t st) {
  if (nctas > 0)
    k_deposit_batch<<<nctas, kBatchQuadThreads, 0, st>>>(desc, cta_rep, thermo, gamma, kT);
}

void launch_deposit_batch_wide(const RepDesc* desc, const int* cta_rep, int nctas,
                               cudaStream_t st) {
  if (nctas > 0) k_deposit_batch_wide<<<nctas, kWideThreads, 0, st>>>(desc, cta_rep);
}

void launch_gather_batch_wide(int prec, const RepDesc* desc, const int* cta_rep, int nctas,
                              int par, int thermo, cudaStream_t st) {
  if (nctas <= 0) return;
  if (prec == 1)
    k_gather_batch_wide<float><<<nctas, kWideThreads, 0, st>>>(desc, cta_rep, par, thermo);
  else
    k_gather_batch_wide<double><<<nctas, kWideThreads, 0, st>>>(desc, cta_rep, par, thermo);
}

void launch_apply_batch(int prec, const RepDesc* desc, const int* cta_rep, int nctas, int par,
                        cudaStream_t st) {
  if (nctas <= 0) return;
  if (prec == 1)
    k_apply_batch<float><<<nctas, kBatchQuadThreads, 0, st>>>(desc, cta_rep, par);
  else
    k_apply_batch<double><<<nctas, kBatchQuadThreads, 0, st>>>(desc, cta_rep, par);
}

void launch_apply_dense_batch(int prec, const RepDesc* desc, const int2* chunk, int nchunks,
                              int par, cudaStream_t st) {
  if (nchunks <= 0) return;
  if (prec == 1)
    k_apply_dense_batch<float><<<nchunks, kApplyThreads, 0, st>>>(desc, chunk, par);
  else
    k_apply_dense_batch<double><<<nchunks, kApplyThreads, 0, st>>>(desc, chunk, par);
}

void launch_gather_batch(int prec, const RepDesc* desc, const int* cta_rep, int nctas, int par,
                         int thermo, double gamma, double kT, cudaStream_t st) {
  if (nctas <= 0) return;
  if (prec == 1)
    k_gather_batch<float><<<nctas, kBatchQuadThreads, 0, st>>>(desc, cta_rep, par, thermo, gamma,
                                                               kT);
  else
    k_gather_batch<double><<<nctas, kBatchQuadThreads, 0, st>>>(desc, cta_rep, par, thermo,
                                                                gamma, kT);
}

void launch_particle_energy(const Mesh& m, const StepParams& sp, Particles p, const double* ie64,
                            double* part_ke, double* part_self, cudaStream_t st) {
  k_particle_energy<<<kRedBlocks, kRedThreads, 0, st>>>(m, sp, p, ie64, part_ke, part_self);
}

}  // namespace memd
