// memd_setup.cu -- create-time and initial-solution kernels of MEMD.
//
//   eps on the links (Sec. II, Fig. 2b)
//   lattice Green's table for the self-energy term (Sec. III, Eqs. 25-27)
//   initial Gauss solution in exact int64 flux (Sec. II, Fig. 1, Eqs. 1-3)
//   deterministic FP64 reductions used by the relaxation and diagnostics
#include "memd_internal.cuh"

namespace memd {

namespace {

constexpr int kThreads = 256;
constexpr int kRedThreads = 256;
constexpr int kRedBlocks = 2 * 152;
constexpr int kGreenBlocks = 152;

inline unsigned blocks_for(int64_t n, int t = kThreads) {
  int64_t b = (n + t - 1) / t;
  return (unsigned)(b < 1 ? 1 : b);
}

__device__ inline void coords(const Mesh& m, int64_t v, int& i, int& j, int& k) {
  i = (int)(v % m.n[0]);
  const int64_t r = v / m.n[0];
  j = (int)(r % m.n[1]);
  k = (int)(r / m.n[1]);
}

// ------------------------------------------------------------------ eps
// A link takes the mean of its end-vertex values; analytic profiles are
// sampled at the link midpoint, with the tanh slab using the periodic
// distance to its centre.
//
// Interface links (Sec. II, Eq. dielectric-interpolation): a link whose end
// values differ across an explicit interface holds the two media in series,
//   1/eps = t / eps1 + (1 - t) / eps2,
// t a the distance from its first end to the interface.  The geometry
// (which side a vertex is on, where a link is cut) is done with explicitly
// rounded operations so that no contraction moves a decision.

// -1 outside, +1 inside, 0 exactly on the interface (takes the mean)
__device__ int slab_side(const Mesh& m, const EpsDesc& e, int k) {
  if (e.p[2] == e.p[3]) return -1;
  const double lo = e.p[2] / m.a, hi = e.p[3] / m.a, u = (double)k;
  if (u == lo || u == hi) return 0;
  return (u > lo && u < hi) ? 1 : -1;
}

// offset of vertex c from the ball's centre in cells, nearest periodic image
__device__ double ball_offset(const Mesh& m, const EpsDesc& e, int c, int d) {
  const double x = __dsub_rn((double)c, e.p[2 + d] / m.a);
  const double n = (double)m.n[d];
  return __dsub_rn(x, __dmul_rn(n, round(x / n)));
}

__device__ int ball_side(const Mesh& m, const EpsDesc& e, const int c[3]) {
  const double r = e.p[5] / m.a;
  const double o0 = ball_offset(m, e, c[0], 0), o1 = ball_offset(m, e, c[1], 1),
               o2 = ball_offset(m, e, c[2], 2);
  const double r2 = __dadd_rn(__dadd_rn(__dmul_rn(o0, o0), __dmul_rn(o1, o1)), __dmul_rn(o2, o2));
  const double rr = __dmul_rn(r, r);
  return r2 < rr ? 1 : (r2 == rr ? 0 : -1);
}

__device__ double medium(const EpsDesc& e, int side) {
  return side > 0 ? e.p[1] : (side < 0 ? e.p[0] : 0.5 * (e.p[0] + e.p[1]));
}

__device__ double clamp_unit(double t) { return t < 0.0 ? 0.0 : (t > 1.0 ? 1.0 : t); }

// 1/eps of link (d, v) for the kinds with values on the vertices or with an
// explicit interface
__device__ double interface_kinds(const Mesh& m, const EpsDesc& e, const double* values, int d,
                                  int64_t v, const int c[3]) {
  int cn[3] = {c[0], c[1], c[2]};
  cn[d] = (cn[d] + 1 == m.n[d]) ? 0 : cn[d] + 1;
  double e1, e2;
  int s1 = 0, s2 = 0;
  if (e.kind == 5 || e.kind == 6) {
    s1 = e.kind == 5 ? slab_side(m, e, c[e.axis]) : ball_side(m, e, c);
    s2 = e.kind == 5 ? slab_side(m, e, cn[e.axis]) : ball_side(m, e, cn);
    e1 = medium(e, s1);
    e2 = medium(e, s2);
  } else {
    e1 = values[v];
    e2 = values[vindex(m, cn[0], cn[1], cn[2])];
  }
  double t = -1.0;
  if (e1 != e2) {
    if (e.kind == 2) {
      const double lo = fmin(e1, e2);
      if (e.p[0] > 0.0 && fabs(e2 - e1) > e.p[0] * lo) t = 0.5;
    } else if (e.kind == 7) {
      const double f = values[m.V + d * m.V + v];
      if (f >= 0.0 && f <= 1.0) t = f;
    } else if (s1 == 0) {
      t = 0.0;
    } else if (s2 == 0) {
      t = 1.0;
    } else if (e.kind == 5) {
      const double face = (s1 < 0 ? e.p[2] : e.p[3]) / m.a;
      t = clamp_unit(__dsub_rn(face, (double)c[d]));
    } else {
      const int d1 = d == 0 ? 1 : 0, d2 = d == 2 ? 1 : 2;
      const double r = e.p[5] / m.a;
      const double od = ball_offset(m, e, c[d], d);
      const double o1 = ball_offset(m, e, c[d1], d1), o2 = ball_offset(m, e, c[d2], d2);
      const double h2 = __dsub_rn(__dmul_rn(r, r), __dadd_rn(__dmul_rn(o1, o1), __dmul_rn(o2, o2)));
      const double h = h2 > 0.0 ? sqrt(h2) : 0.0;
      t = clamp_unit(s1 > 0 ? __dadd_rn(-od, h) : __dsub_rn(-od, h));
    }
  }
  if (t < 0.0) return 1.0 / (0.5 * (e1 + e2));
  return t / e1 + (1.0 - t) / e2;
}

__global__ void k_eps_links(Mesh m, EpsDesc e, const double* __restrict__ values,
                            double* __restrict__ ie, unsigned int* err) {
  const int64_t V = m.V;
  const int64_t l = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (l >= 3 * V) return;
  const int d = (int)(l / V);
  const int64_t v = l - d * V;
  int c[3];
  coords(m, v, c[0], c[1], c[2]);
  double eps = 0.0;
  switch (e.kind) {
    case 0:
      eps = e.p[0];
      break;
    case 1:
      eps = values[l];
      break;
    case 2:
    case 5:
    case 6:
    case 7: {
      const double inv = interface_kinds(m, e, values, d, v, c);
      eps = 1.0 / inv;
      if (eps > 0.0 && isfinite(eps) && isfinite(inv)) {
        ie[l] = inv;
        return;
      }
      break;
    }
    case 3:
    case 4: {
      const int ax = e.axis;
      double s = (double)c[ax] * m.a;
      if (d == ax) s += 0.5 * m.a;
      const double Lx = m.L[ax];
      if (e.kind == 3) {
        double dz = s - e.p[2];
        dz = dz - Lx * round(dz / Lx);
        eps = e.p[0] + e.p[1] * tanh((fabs(dz) - e.p[3]) / e.p[4]);
      } else {
        eps = e.p[0] + e.p[1] * sin(2.0 * 3.141592653589793 * s / Lx + e.p[2]);
      }
      break;
    }
    default:
      eps = -1.0;
  }
  if (!(eps > 0.0) || !isfinite(eps)) {
    atomicOr(err, kErrNonFinite);
    eps = 1.0;
  }
  ie[l] = 1.0 / eps;
}

template <typename T>
__global__ void k_cast(T* __restrict__ dst, const double* __restrict__ src, int64_t n) {
  const int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (t < n) dst[t] = (T)src[t];
}

template <typename T>
__global__ void k_widen(double* __restrict__ dst, const T* __restrict__ src, int64_t n) {
  const int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (t < n) dst[t] = (double)src[t];
}

// --------------------------------------------------------- Green's table
// G(r) = (1/V) sum_{k != 0} cos(k.r) / sum_d 4 sin^2(k_d/2) for the 8
// displacements r in {0,1}^3; block partial sums over a fixed mode split,
// then a fixed-order final sum.
__global__ void __launch_bounds__(kThreads) k_green_partial(Mesh m, double* __restrict__ part) {
  __shared__ double sh[8][kThreads / 32];
  double acc[8];
  for (int t = 0; t < 8; ++t) acc[t] = 0.0;
  const double tpi = 2.0 * 3.141592653589793;
  for (int64_t g = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; g < m.V;
       g += (int64_t)gridDim.x * blockDim.x) {
    if (g == 0) continue;
    int mx, my, mz;
    coords(m, g, mx, my, mz);
    const double kx = tpi * mx / m.n[0], ky = tpi * my / m.n[1], kz = tpi * mz / m.n[2];
    const double sx = sin(0.5 * kx), sy = sin(0.5 * ky), sz = sin(0.5 * kz);
    const double inv = 1.0 / (4.0 * (sx * sx + sy * sy + sz * sz));
    const double cx = cos(kx), cy = cos(ky), cz = cos(kz);
    const double snx = sin(kx), sny = sin(ky), snz = sin(kz);
    // cos(k.r) for r in {0,1}^3 from the angle-sum identities
    const double cxy = cx * cy - snx * sny, sxy = snx * cy + cx * sny;
    acc[0] += inv;
    acc[1] += cx * inv;
    acc[2] += cy * inv;
    acc[3] += cxy * inv;
    acc[4] += cz * inv;
    acc[5] += (cx * cz - snx * snz) * inv;
    acc[6] += (cy * cz - sny * snz) * inv;
    acc[7] += (cxy * cz - sxy * snz) * inv;
  }
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  for (int t = 0; t < 8; ++t) {
    double x = acc[t];
    for (int o = 16; o > 0; o >>= 1) x += __shfl_down_sync(0xffffffffu, x, o);
    if (lane == 0) sh[t][w] = x;
  }
  __syncthreads();
  if (threadIdx.x < 8) {
    double s = 0.0;
    for (int q = 0; q < kThreads / 32; ++q) s += sh[threadIdx.x][q];
    part[blockIdx.x * 8 + threadIdx.x] = s;
  }
}

__global__ void k_green_final(Mesh m, const double* __restrict__ part, double* __restrict__ G) {
  const int t = threadIdx.x;
  if (t >= 8) return;
  double s = 0.0;
  for (int b = 0; b < kGreenBlocks; ++b) s += part[b * 8 + t];
  G[t] = s / (double)m.V;
}

// -------------------------------------------------------------- Gauss scan
__device__ inline long long floordiv(long long a, long long b) {
  long long q = a / b;
  if ((a % b != 0) && ((a < 0) != (b < 0))) --q;
  return q;
}

// share t of F split over M links: floor(F/M), plus one on the first F mod M
__device__ inline long long share(long long F, long long M, long long t) {
  const long long base = floordiv(F, M);
  const long long rem = F - base * M;
  return base + (t < rem ? 1 : 0);
}

__device__ inline long long block_sum_ll(long long x, long long* sh) {
  for (int o = 16; o > 0; o >>= 1) x += __shfl_down_sync(0xffffffffu, x, o);
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  if (lane == 0) sh[w] = x;
  __syncthreads();
  long long r = 0;
  if (threadIdx.x == 0)
    for (int t = 0; t < (int)(blockDim.x >> 5); ++t) r += sh[t];
  __syncthreads();
  return r;
}

// rho[k] = sum of Q over plane k (one block per plane)
__global__ void __launch_bounds__(kThreads)
    k_plane_sums(Mesh m, const long long* __restrict__ Q, long long* __restrict__ rho) {
  __shared__ long long sh[kThreads / 32];
  const int64_t P = (int64_t)m.n[0] * m.n[1];
  const int k = blockIdx.x;
  long long s = 0;
  for (int64_t t = threadIdx.x; t < P; t += blockDim.x) s += Q[t + P * k];
  s = block_sum_ll(s, sh);
  if (threadIdx.x == 0) rho[k] = s;
}

// cumulative plane charge F[k] = rho[0] + ... + rho[k]; must close at zero
__global__ void k_prefix(const long long* __restrict__ rho, long long* __restrict__ F, int n,
                         unsigned int* err) {
  if (threadIdx.x != 0 || blockIdx.x != 0) return;
  long long s = 0;
  for (int k = 0; k < n; ++k) {
    s += rho[k];
    F[k] = s;
  }
  if (s != 0) atomicOr(err, kErrGauss);
}

// z-links of plane k carry share(F[k]); the residual charge stays on the vertices
__global__ void k_zflux(Mesh m, const long long* __restrict__ Q, const long long* __restrict__ F,
                        long long* __restrict__ Lg, long long* __restrict__ r) {
  const int64_t v = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (v >= m.V) return;
  const int64_t P = (int64_t)m.n[0] * m.n[1];
  const int k = (int)(v / P);
  const int64_t t = v - (int64_t)k * P;
  const long long out = share(F[k], P, t);
  const long long in = (k == 0) ? 0 : share(F[k - 1], P, t);
  Lg[kLT * tl_pair(2, v)] = out;
  r[v] = Q[v] - (out - in);
}

// lam[j + ny k] = sum of r over the y-line (j, k) (one warp per line)
__global__ void k_line_sums(Mesh m, const long long* __restrict__ r, long long* __restrict__ lam) {
  const int64_t line = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
  const int lane = threadIdx.x & 31;
  const int64_t nl = (int64_t)m.n[1] * m.n[2];
  if (line >= nl) return;
  long long s = 0;
  for (int i = lane; i < m.n[0]; i += 32) s += r[line * m.n[0] + i];
  for (int o = 16; o > 0; o >>= 1) s += __shfl_down_sync(0xffffffffu, s, o);
  if (lane == 0) lam[line] = s;
}

// per plane: Fy[j, k] = lam[0, k] + ... + lam[j, k]; must close at zero
__global__ void k_line_prefix(Mesh m, const long long* __restrict__ lam, long long* __restrict__ Fy,
                              unsigned int* err) {
  const int k = blockIdx.x * blockDim.x + threadIdx.x;
  if (k >= m.n[2]) return;
  long long s = 0;
  for (int j = 0; j < m.n[1]; ++j) {
    s += lam[j + (int64_t)m.n[1] * k];
    Fy[j + (int64_t)m.n[1] * k] = s;
  }
  if (s != 0) atomicOr(err, kErrGauss);
}

__global__ void k_yflux(Mesh m, const long long* __restrict__ Fy, long long* __restrict__ Lg,
                        long long* __restrict__ r) {
  const int64_t v = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (v >= m.V) return;
  const int i = (int)(v % m.n[0]);
  const int64_t line = v / m.n[0];  // j + ny k
  const int j = (int)(line % m.n[1]);
  const long long out = share(Fy[line], m.n[0], i);
  const long long in = (j == 0) ? 0 : share(Fy[line - 1], m.n[0], i);
  Lg[kLT * tl_pair(1, v)] = out;
  r[v] -= out - in;
}

// x-links: running sum of the residual along each x-line; must close at zero
__global__ void k_xscan(Mesh m, const long long* __restrict__ r, long long* __restrict__ Lg,
                        unsigned int* err) {
  const int64_t line = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (line >= (int64_t)m.n[1] * m.n[2]) return;
  long long s = 0;
  for (int i = 0; i < m.n[0]; ++i) {
    s += r[line * m.n[0] + i];
    Lg[kLT * tl_pair(0, line * m.n[0] + i)] = s;
  }
  if (s != 0) atomicOr(err, kErrGauss);
}

// zero every kLT-th word of count pairs (the transfer words, leaving the
// ledger words between them)
__global__ void k_clear_transfers(long long* __restrict__ T, int64_t count) {
  for (int64_t l = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; l < count;
       l += (int64_t)gridDim.x * blockDim.x)
    T[kLT * l] = 0;
}

// per-component ledger sums (exact int64)
__global__ void __launch_bounds__(kThreads)
    k_ledger_sums(Mesh m, const long long* __restrict__ Lg, DevState* ds) {
  __shared__ long long sh[kThreads / 32];
  const int d = blockIdx.y;
  long long s = 0;
  for (int64_t v = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; v < m.V;
       v += (int64_t)gridDim.x * blockDim.x)
    s += Lg[kLT * tl_pair(d, v)];
  s = block_sum_ll(s, sh);
  if (threadIdx.x == 0) atomicAdd((unsigned long long*)&ds->lsum[d], (unsigned long long)s);
}

// D = Lg 2^-48/a^2 + shift_d, shift_d = -P_d / Vbox - mean(Lg_d) 2^-48/a^2
__global__ void k_init_D(Mesh m, double* __restrict__ D, const long long* __restrict__ Lg,
                         const DevState* ds, double scale, double Vbox) {
  const int64_t l = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (l >= 3 * m.V) return;
  const int d = (int)(l / m.V);
  const double P = (double)(long long)ds->Pacc[d] * (m.a / (double)kS);
  const double shift = -P / Vbox - ((double)ds->lsum[d] * scale) / (double)m.V;
  D[l] = (double)Lg[kLT * tl_pair(d, l - d * m.V)] * scale + shift;
}

// ------------------------------------------------------------- reductions
__device__ inline double block_sum_d(double x, double* sh) {
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

__device__ inline double block_max_d(double x, double* sh) {
  for (int o = 16; o > 0; o >>= 1) x = fmax(x, __shfl_down_sync(0xffffffffu, x, o));
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  if (lane == 0) sh[w] = x;
  __syncthreads();
  double r = 0.0;
  if (threadIdx.x == 0)
    for (int t = 0; t < (int)(blockDim.x >> 5); ++t) r = fmax(r, sh[t]);
  __syncthreads();
  return r;
}

__global__ void __launch_bounds__(kRedThreads)
    k_dot(const double* __restrict__ x, const double* __restrict__ y, int64_t n,
          double* __restrict__ part) {
  __shared__ double sh[kRedThreads / 32];
  double s = 0.0;
  for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < n;
       t += (int64_t)gridDim.x * blockDim.x)
    s += y ? x[t] * y[t] : x[t];
  s = block_sum_d(s, sh);
  if (threadIdx.x == 0) part[blockIdx.x] = s;
}

__global__ void __launch_bounds__(kRedThreads)
    k_absmax(const double* __restrict__ x, const double* __restrict__ y, int64_t n,
             double* __restrict__ part) {
  __shared__ double sh[kRedThreads / 32];
  double s = 0.0;
  for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < n;
       t += (int64_t)gridDim.x * blockDim.x)
    s = fmax(s, fabs(y ? x[t] * y[t] : x[t]));
  s = block_max_d(s, sh);
  if (threadIdx.x == 0) part[blockIdx.x] = s;
}

__global__ void __launch_bounds__(kRedThreads)
    k_finish(const double* __restrict__ part, int op, double* __restrict__ out) {
  __shared__ double sh[kRedThreads / 32];
  double s = 0.0;
  for (int t = threadIdx.x; t < kRedBlocks; t += blockDim.x)
    s = op ? fmax(s, part[t]) : s + part[t];
  s = op ? block_max_d(s, sh) : block_sum_d(s, sh);
  if (threadIdx.x == 0) out[0] = s;
}

}  // namespace

void launch_eps_links(const Mesh& m, const EpsDesc& e, const double* values, double* ie64,
                      unsigned int* err, cudaStream_t st) {
  k_eps_links<<<blocks_for(3 * m.V), kThreads, 0, st>>>(m, e, values, ie64, err);
}

void launch_cast(int prec, void* dst, const double* src, int64_t count, cudaStream_t st) {
  if (prec == 1)
    k_cast<float><<<blocks_for(count), kThreads, 0, st>>>((float*)dst, src, count);
  else
    cudaMemcpyAsync(dst, src, count * sizeof(double), cudaMemcpyDeviceToDevice, st);
}

void launch_widen(int prec, double* dst, const void* src, int64_t count, cudaStream_t st) {
  if (prec == 1)
    k_widen<float><<<blocks_for(count), kThreads, 0, st>>>(dst, (const float*)src, count);
  else
    cudaMemcpyAsync(dst, src, count * sizeof(double), cudaMemcpyDeviceToDevice, st);
}

int green_partials() { return kGreenBlocks * 8; }

void launch_green(const Mesh& m, double* partial, double* G, cudaStream_t st) {
  k_green_partial<<<kGreenBlocks, kThreads, 0, st>>>(m, partial);
  k_green_final<<<1, 32, 0, st>>>(m, partial, G);
}

int64_t scan_scratch(const Mesh& m) {
  // r (V) + rho (nz) + F (nz) + lam (ny nz) + Fy (ny nz)
  return m.V + 2 * (int64_t)m.n[2] + 2 * (int64_t)m.n[1] * m.n[2];
}

void launch_gauss_scan(const Mesh& m, const long long* Q, long long* Lg, long long* scratch,
                       unsigned int* err, cudaStream_t st) {
  long long* r = scratch;
  long long* rho = r + m.V;
  long long* F = rho + m.n[2];
  long long* lam = F + m.n[2];
  long long* Fy = lam + (int64_t)m.n[1] * m.n[2];
  const int64_t nl = (int64_t)m.n[1] * m.n[2];
  k_plane_sums<<<m.n[2], kThreads, 0, st>>>(m, Q, rho);
  k_prefix<<<1, 32, 0, st>>>(rho, F, m.n[2], err);
  k_zflux<<<blocks_for(m.V), kThreads, 0, st>>>(m, Q, F, Lg, r);
  k_line_sums<<<blocks_for(nl * 32), kThreads, 0, st>>>(m, r, lam);
  k_line_prefix<<<blocks_for(m.n[2], 64), 64, 0, st>>>(m, lam, Fy, err);
  k_yflux<<<blocks_for(m.V), kThreads, 0, st>>>(m, Fy, Lg, r);
  k_xscan<<<blocks_for(nl, 128), 128, 0, st>>>(m, r, Lg, err);
}

// ------------------------------------------- permittivity from salt density
// |q| density in e at the vertices from its fixed-point deposit
__global__ void k_density_from_ll(int64_t V, const long long* __restrict__ Q,
                                  double* __restrict__ rho) {
  const int64_t v = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (v < V) rho[v] = __dmul_rn((double)Q[v], 3.552713678800501e-15);  // 2^-48
}

// one axis of the periodic Gaussian smoothing: out(v) = sum_{j=-R..R} w_j
// in(v + j e_axis), summed in order of j, every product and sum rounded
// on its own (the same roundings as a plain sequential loop)
__global__ void k_smooth_axis(Mesh m, const double* __restrict__ in, double* __restrict__ out,
                              int axis, const double* __restrict__ w, int R) {
  const int64_t v = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (v >= m.V) return;
  int c[3];
  coords(m, v, c[0], c[1], c[2]);
  const int n = m.n[axis];
  double acc = 0.0;
  for (int j = -R; j <= R; ++j) {
    int e[3] = {c[0], c[1], c[2]};
    e[axis] = ((e[axis] + j) % n + n) % n;
    acc = __dadd_rn(acc, __dmul_rn(w[j + R], in[vindex(m, e[0], e[1], e[2])]));
  }
  out[v] = acc;
}

// eps(v) = eps0 + slope (rho(v) / mean - 1) clamped to [lo, hi]; mean[0]
// holds the sum of rho over the V vertices
__global__ void k_salt_map(int64_t V, const double* __restrict__ rho, const double* __restrict__ sum,
                           double eps0, double slope, double lo, double hi,
                           double* __restrict__ eps) {
  const int64_t v = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (v >= V) return;
  const double mean = __ddiv_rn(sum[0], (double)V);
  double e = eps0;
  if (mean > 0.0)
    e = __dadd_rn(eps0, __dmul_rn(slope, __dsub_rn(__ddiv_rn(rho[v], mean), 1.0)));
  eps[v] = e < lo ? lo : (e > hi ? hi : e);
}

void launch_salt_eps(const Mesh& m, const long long* Q, double* rho, double* tmp,
                     const double* w, int R, double sigma, double* part, double* sum,
                     const double rule[4], double* eps, cudaStream_t st) {
  const unsigned nb = (unsigned)((m.V + 255) / 256);
  k_density_from_ll<<<nb, 256, 0, st>>>(m.V, Q, rho);
  if (sigma > 0.0) {
    // x, then y, then z (ping-pong through tmp; the result back in rho)
    k_smooth_axis<<<nb, 256, 0, st>>>(m, rho, tmp, 0, w, R);
    k_smooth_axis<<<nb, 256, 0, st>>>(m, tmp, rho, 1, w, R);
    k_smooth_axis<<<nb, 256, 0, st>>>(m, rho, tmp, 2, w, R);
    cudaMemcpyAsync(rho, tmp, sizeof(double) * m.V, cudaMemcpyDeviceToDevice, st);
  }
  launch_dot(rho, nullptr, m.V, part, st);
  launch_finish(part, 0, sum, st);
  k_salt_map<<<nb, 256, 0, st>>>(m.V, rho, sum, rule[0], rule[1], rule[2], rule[3], eps);
}

void launch_clear_transfers(long long* T, int64_t count, cudaStream_t st) {
  if (count > 0) k_clear_transfers<<<2 * 152, 256, 0, st>>>(T, count);
}

void launch_ledger_sums(const Mesh& m, const long long* Lg, DevState* ds, cudaStream_t st) {
  cudaMemsetAsync(ds->lsum, 0, sizeof(ds->lsum), st);
  k_ledger_sums<<<dim3(kRedBlocks, 3, 1), kThreads, 0, st>>>(m, Lg, ds);
}

void launch_init_D(const Mesh& m, double* D64, const long long* Lg, DevState* ds, double scale,
                   double Vbox, cudaStream_t st) {
  k_init_D<<<blocks_for(3 * m.V), kThreads, 0, st>>>(m, D64, Lg, ds, scale, Vbox);
}

int reduce_blocks() { return kRedBlocks; }

void launch_dot(const double* x, const double* y, int64_t n, double* partial, cudaStream_t st) {
  k_dot<<<kRedBlocks, kRedThreads, 0, st>>>(x, y, n, partial);
}

void launch_absmax(const double* x, const double* y, int64_t n, double* partial,
                   cudaStream_t st) {
  k_absmax<<<kRedBlocks, kRedThreads, 0, st>>>(x, y, n, partial);
}

void launch_finish(const double* partial, int op, double* out, cudaStream_t st) {
  k_finish<<<1, kRedThreads, 0, st>>>(partial, op, out);
}

}  // namespace memd
