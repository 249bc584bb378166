// memd_mg.cu -- the initial field and the effective permittivity through a
// scalar potential (Sec. II and Sec. V).
//
// The relaxed field is the minimiser of sum D^2 / 2 eps at fixed div D and
// fixed mean of D; at the minimum E = D / eps is curl free, i.e. a lattice
// gradient plus a constant: D = eps (-grad phi + E0).  phi solves the
// variable-coefficient Poisson problem L phi = -div(eps grad phi) = f on the
// periodic vertex lattice, and E0 follows from the mean of D through the
// effective permittivity, whose columns come from the three cell problems
// L psi_d = -div(eps e_d) (homogenisation).  The plaquette-rotation
// relaxation reaches the same minimiser; this is a faster route to it on
// V unknowns instead of 3V.
//
// Solver: conjugate gradients preconditioned by one symmetric multigrid
// V-cycle.  A level whose extents are all even coarsens geometrically
// (vertex-centred, by 2): red-black Gauss-Seidel, full-weighting
// restriction, trilinear prolongation, coarse link conductances from two
// fine links in series averaged over the 3 x 3 perpendicular neighbourhood.
// A level with an odd extent coarsens by aggregating vertex pairs (a triple
// at the end of an odd axis): damped Jacobi, Galerkin coarse operator,
// piecewise-constant transfers with an over-corrected coarse correction.
// FP64 throughout.
#include <algorithm>
#include <cmath>
#include <vector>

#include "memd_ctx.cuh"
#include "memd_internal.cuh"

namespace memd {

namespace {

constexpr int kT = 256;
inline unsigned nblk(int64_t n) { return (unsigned)((n + kT - 1) / kT); }

struct Lv {
  int n0, n1, n2;
  int64_t V;
};

__device__ __forceinline__ int wrp(int i, int n) { return i < 0 ? i + n : (i >= n ? i - n : i); }

__device__ __forceinline__ void coords(const Lv& L, int64_t v, int& i, int& j, int& k) {
  i = (int)(v % L.n0);
  const int64_t t = v / L.n0;
  j = (int)(t % L.n1);
  k = (int)(t / L.n1);
}

__device__ __forceinline__ int64_t vid(const Lv& L, int i, int j, int k) {
  return (int64_t)i + (int64_t)L.n0 * ((int64_t)j + (int64_t)L.n1 * k);
}

// (L phi)(v) and the diagonal: sum over the 6 links at v of w (phi_v - phi_nb)
__device__ __forceinline__ double apply_at(const Lv& L, const double* __restrict__ w,
                                           const double* __restrict__ phi, int64_t v, int i,
                                           int j, int k, double& nbsum, double& dg) {
  const int64_t V = L.V;
  const int64_t xp = vid(L, wrp(i + 1, L.n0), j, k), xm = vid(L, wrp(i - 1, L.n0), j, k);
  const int64_t yp = vid(L, i, wrp(j + 1, L.n1), k), ym = vid(L, i, wrp(j - 1, L.n1), k);
  const int64_t zp = vid(L, i, j, wrp(k + 1, L.n2)), zm = vid(L, i, j, wrp(k - 1, L.n2));
  const double wxp = w[v], wxm = w[xm], wyp = w[V + v], wym = w[V + ym], wzp = w[2 * V + v],
               wzm = w[2 * V + zm];
  dg = ((wxp + wxm) + (wyp + wym)) + (wzp + wzm);
  nbsum = ((wxp * phi[xp] + wxm * phi[xm]) + (wyp * phi[yp] + wym * phi[ym])) +
          (wzp * phi[zp] + wzm * phi[zm]);
  return dg * phi[v] - nbsum;
}

__global__ void k_residual(Lv L, const double* __restrict__ w, const double* __restrict__ phi,
                           const double* __restrict__ f, double* __restrict__ r) {
  const int64_t v = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (v >= L.V) return;
  int i, j, k;
  coords(L, v, i, j, k);
  double nb, dg;
  const double a = apply_at(L, w, phi, v, i, j, k, nb, dg);
  r[v] = (f ? f[v] : 0.0) - a;
}

// q = L p
__global__ void k_apply(Lv L, const double* __restrict__ w, const double* __restrict__ p,
                        double* __restrict__ q) {
  const int64_t v = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (v >= L.V) return;
  int i, j, k;
  coords(L, v, i, j, k);
  double nb, dg;
  q[v] = apply_at(L, w, p, v, i, j, k, nb, dg);
}

// Gauss-Seidel on the vertices of one colour ((i + j + k) mod 2)
__global__ void k_rbgs(Lv L, const double* __restrict__ w, double* __restrict__ phi,
                       const double* __restrict__ f, int color) {
  const int64_t h = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;  // half-index
  const int64_t v0 = 2 * h;
  if (v0 >= L.V) return;
  // every x row has an even length: the vertex of this colour is v0 or v0+1
  int i, j, k;
  coords(L, v0, i, j, k);
  int64_t v = v0;
  if (((i + j + k) & 1) != color) {
    v = v0 + 1;
    i += 1;
  }
  double nb, dg;
  apply_at(L, w, phi, v, i, j, k, nb, dg);
  phi[v] = (f[v] + nb) / dg;
}

// damped Jacobi: phi += omega (f - L phi) / diag, in two passes through r
__global__ void k_jacobi_res(Lv L, const double* __restrict__ w, const double* __restrict__ phi,
                             const double* __restrict__ f, double* __restrict__ r) {
  const int64_t v = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (v >= L.V) return;
  int i, j, k;
  coords(L, v, i, j, k);
  double nb, dg;
  const double a = apply_at(L, w, phi, v, i, j, k, nb, dg);
  r[v] = (f[v] - a) / dg;
}

__global__ void k_jacobi_upd(int64_t V, double* __restrict__ phi, const double* __restrict__ r,
                             double omega) {
  const int64_t v = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (v < V) phi[v] += omega * r[v];
}

// full weighting: fc(I) = sum_o prod_d (1 - |o_d| / 2) / 8 r(2 I + o)
__global__ void k_restrict(Lv F, Lv Cc, const double* __restrict__ r, double* __restrict__ fc) {
  const int64_t V = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (V >= Cc.V) return;
  int I, J, K;
  coords(Cc, V, I, J, K);
  double s = 0.0;
  for (int oz = -1; oz <= 1; ++oz)
    for (int oy = -1; oy <= 1; ++oy)
      for (int ox = -1; ox <= 1; ++ox) {
        const double wt = (ox ? 0.5 : 1.0) * (oy ? 0.5 : 1.0) * (oz ? 0.5 : 1.0);
        s += wt * r[vid(F, wrp(2 * I + ox, F.n0), wrp(2 * J + oy, F.n1), wrp(2 * K + oz, F.n2))];
      }
  fc[V] = 0.125 * s;
}

// trilinear prolongation of the coarse correction, added to phi
__global__ void k_prolong(Lv F, Lv Cc, const double* __restrict__ ec, double* __restrict__ phi) {
  const int64_t v = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (v >= F.V) return;
  int i, j, k;
  coords(F, v, i, j, k);
  const int I0 = i >> 1, J0 = j >> 1, K0 = k >> 1;
  const int di = i & 1, dj = j & 1, dk = k & 1;
  double s = 0.0;
  for (int c = 0; c < 8; ++c) {
    const int ax = c & 1, ay = (c >> 1) & 1, az = c >> 2;
    if ((ax && !di) || (ay && !dj) || (az && !dk)) continue;
    const double wt = (di ? 0.5 : 1.0) * (dj ? 0.5 : 1.0) * (dk ? 0.5 : 1.0);
    s += wt * ec[vid(Cc, wrp(I0 + ax, Cc.n0), wrp(J0 + ay, Cc.n1), wrp(K0 + az, Cc.n2))];
  }
  phi[v] += s;
}

// coarse conductance of link (d, I): the two fine d-links from 2I + o (o
// perpendicular to d) in series, averaged with weights (1/4, 1/2, 1/4)^2
// over o, halved for the coarse spacing
__global__ void k_coarsen(Lv F, Lv Cc, const double* __restrict__ wf, double* __restrict__ wc) {
  const int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (t >= 3 * Cc.V) return;
  const int d = (int)(t / Cc.V);
  const int64_t V = t - (int64_t)d * Cc.V;
  int I, J, K;
  coords(Cc, V, I, J, K);
  const int e1 = (d + 1) % 3, e2 = (d + 2) % 3;
  double s = 0.0;
  for (int b = -1; b <= 1; ++b)
    for (int a = -1; a <= 1; ++a) {
      int p[3] = {2 * I, 2 * J, 2 * K};
      p[e1] += a;
      p[e2] += b;
      int q[3] = {p[0], p[1], p[2]};
      q[d] += 1;
      const int64_t l1 = (int64_t)d * F.V + vid(F, wrp(p[0], F.n0), wrp(p[1], F.n1), wrp(p[2], F.n2));
      const int64_t l2 = (int64_t)d * F.V + vid(F, wrp(q[0], F.n0), wrp(q[1], F.n1), wrp(q[2], F.n2));
      const double w1 = wf[l1], w2 = wf[l2];
      const double ser = w1 * w2 / (w1 + w2);
      s += (a ? 0.5 : 1.0) * (b ? 0.5 : 1.0) * 0.25 * ser;
    }
  wc[t] = 0.5 * s;
}

// Aggregation (a level with an odd extent): coarse vertex I along an axis
// of n fine vertices and m = n / 2 coarse ones holds fine 2I, 2I + 1, and
// also 2I + 2 when it is the last one of an odd n.  Piecewise-constant
// prolongation; the Galerkin coarse operator is the aggregates' graph
// Laplacian, the conductance of coarse link (d, I) the sum of the fine
// d-links leaving aggregate I towards I + e_d.
__device__ __forceinline__ int agg_lo(int I) { return 2 * I; }
__device__ __forceinline__ int agg_hi(int I, int m, int n) { return I == m - 1 ? n - 1 : 2 * I + 1; }
__device__ __forceinline__ int agg_of(int i, int m) { return min(i >> 1, m - 1); }

__global__ void k_agg_coarsen(Lv F, Lv Cc, const double* __restrict__ wf, double* __restrict__ wc) {
  const int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (t >= 3 * Cc.V) return;
  const int d = (int)(t / Cc.V);
  const int64_t V = t - (int64_t)d * Cc.V;
  int C[3];
  coords(Cc, V, C[0], C[1], C[2]);
  const int nf[3] = {F.n0, F.n1, F.n2}, nc[3] = {Cc.n0, Cc.n1, Cc.n2};
  int lo[3], hi[3];
  for (int e = 0; e < 3; ++e) {
    lo[e] = agg_lo(C[e]);
    hi[e] = agg_hi(C[e], nc[e], nf[e]);
  }
  lo[d] = hi[d];  // the last fine layer of the aggregate along d
  double s = 0.0;
  for (int k = lo[2]; k <= hi[2]; ++k)
    for (int j = lo[1]; j <= hi[1]; ++j)
      for (int i = lo[0]; i <= hi[0]; ++i) s += wf[(int64_t)d * F.V + vid(F, i, j, k)];
  wc[t] = s;
}

__global__ void k_agg_restrict(Lv F, Lv Cc, const double* __restrict__ r, double* __restrict__ fc) {
  const int64_t V = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (V >= Cc.V) return;
  int I, J, K;
  coords(Cc, V, I, J, K);
  const int i1 = agg_hi(I, Cc.n0, F.n0), j1 = agg_hi(J, Cc.n1, F.n1), k1 = agg_hi(K, Cc.n2, F.n2);
  double s = 0.0;
  for (int k = agg_lo(K); k <= k1; ++k)
    for (int j = agg_lo(J); j <= j1; ++j)
      for (int i = agg_lo(I); i <= i1; ++i) s += r[vid(F, i, j, k)];
  fc[V] = s;
}

// phi += alpha e(aggregate of v); alpha > 1 makes up for the flat prolongation
__global__ void k_agg_prolong(Lv F, Lv Cc, const double* __restrict__ ec, double alpha,
                              double* __restrict__ phi) {
  const int64_t v = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (v >= F.V) return;
  int i, j, k;
  coords(F, v, i, j, k);
  phi[v] += alpha * ec[vid(Cc, agg_of(i, Cc.n0), agg_of(j, Cc.n1), agg_of(k, Cc.n2))];
}

// The coarsest level (at most kCoarseSmem vertices) in one CTA: sweeps
// forward (red then black, or damped Jacobi) then backward, all in shared
// memory, instead of one launch per half-sweep.
constexpr int kCoarseSmem = 1024;

__global__ void __launch_bounds__(1024)
    k_coarse_solve(Lv L, const double* __restrict__ w, const double* __restrict__ f,
                   double* __restrict__ phi, int sweeps, int rb) {
  extern __shared__ double sm[];
  const int V = (int)L.V;
  double* sw = sm;            // 3V
  double* sf = sm + 3 * V;    // V
  double* sp = sm + 4 * V;    // V
  double* st = sm + 5 * V;    // V
  for (int t = threadIdx.x; t < 3 * V; t += blockDim.x) sw[t] = w[t];
  for (int t = threadIdx.x; t < V; t += blockDim.x) {
    sf[t] = f[t];
    sp[t] = 0.0;
  }
  __syncthreads();
  auto relax_vertex = [&](int v, bool jac) {
    int i, j, k;
    coords(L, v, i, j, k);
    double nb, dg;
    const double a = apply_at(L, sw, sp, v, i, j, k, nb, dg);
    if (jac)
      st[v] = (sf[v] - a) / dg;
    else
      sp[v] = (sf[v] + nb) / dg;
  };
  for (int dir = 0; dir < 2; ++dir)
    for (int s = 0; s < sweeps; ++s) {
      if (rb) {
        for (int h = 0; h < 2; ++h) {
          const int color = dir == 0 ? h : 1 - h;
          for (int v = threadIdx.x; v < V; v += blockDim.x) {
            int i, j, k;
            coords(L, v, i, j, k);
            if (((i + j + k) & 1) == color) relax_vertex(v, false);
          }
          __syncthreads();
        }
      } else {
        for (int v = threadIdx.x; v < V; v += blockDim.x) relax_vertex(v, true);
        __syncthreads();
        for (int v = threadIdx.x; v < V; v += blockDim.x) sp[v] += 0.8 * st[v];
        __syncthreads();
      }
    }
  for (int t = threadIdx.x; t < V; t += blockDim.x) phi[t] = sp[t];
}

// fine conductances w = eps / a^2 = 1 / (ie a^2)
__global__ void k_fine_w(int64_t n, const double* __restrict__ ie64, double inv_a2,
                         double* __restrict__ w) {
  const int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (t < n) w[t] = inv_a2 / ie64[t];
}

// f = div F (links -> vertices), F given as 3V link values, scaled by s
__global__ void k_div_links(Lv L, const double* __restrict__ F, double s, double* __restrict__ f) {
  const int64_t v = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (v >= L.V) return;
  int i, j, k;
  coords(L, v, i, j, k);
  const int64_t V = L.V;
  const double dx = F[v] - F[vid(L, wrp(i - 1, L.n0), j, k)];
  const double dy = F[V + v] - F[V + vid(L, i, wrp(j - 1, L.n1), k)];
  const double dz = F[2 * V + v] - F[2 * V + vid(L, i, j, wrp(k - 1, L.n2))];
  f[v] = s * ((dx + dy) + dz);
}

// f = -div(eps e_d) = -(eps_d(v) - eps_d(v - e_d)) / a
__global__ void k_div_eps_unit(Lv L, const double* __restrict__ ie64, int d, double inv_a,
                               double* __restrict__ f) {
  const int64_t v = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (v >= L.V) return;
  int i, j, k;
  coords(L, v, i, j, k);
  int c[3] = {i, j, k};
  c[d] -= 1;
  const int64_t vm = vid(L, wrp(c[0], L.n0), wrp(c[1], L.n1), wrp(c[2], L.n2));
  f[v] = -(1.0 / ie64[(int64_t)d * L.V + v] - 1.0 / ie64[(int64_t)d * L.V + vm]) * inv_a;
}

// out = eps (g e_dir - grad phi) on every link, scaled: out_e(v) = eps_e(v) *
// (g [e == dir] - (phi(v + e_e) - phi(v)) / a); dir < 0 for no constant
__global__ void k_flux(Lv L, const double* __restrict__ ie64, const double* __restrict__ phi,
                       int dir, double g, double inv_a, double* __restrict__ out, int accumulate,
                       double scale) {
  const int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (t >= 3 * L.V) return;
  const int e = (int)(t / L.V);
  const int64_t v = t - (int64_t)e * L.V;
  int i, j, k;
  coords(L, v, i, j, k);
  int c[3] = {i, j, k};
  c[e] += 1;
  const int64_t vp = vid(L, wrp(c[0], L.n0), wrp(c[1], L.n1), wrp(c[2], L.n2));
  const double val = ((e == dir ? g : 0.0) - (phi[vp] - phi[v]) * inv_a) / ie64[t];
  out[t] = accumulate ? out[t] + scale * val : scale * val;
}

// CG scalars on the device: s[0] = p.q, s[1] = r.z (old), s[2] = r.z (new)
__global__ void k_cg_xr(int64_t n, double* __restrict__ x, double* __restrict__ r,
                        const double* __restrict__ p, const double* __restrict__ q,
                        const double* __restrict__ s, int rz) {
  const int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (t >= n) return;
  const double pq = s[0];
  const double alpha = pq != 0.0 ? s[rz] / pq : 0.0;
  x[t] += alpha * p[t];
  r[t] -= alpha * q[t];
}

__global__ void k_cg_p(int64_t n, double* __restrict__ p, const double* __restrict__ z,
                       const double* __restrict__ s, int rz_new, int rz_old) {
  const int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (t >= n) return;
  const double b = s[rz_old];
  const double beta = b != 0.0 ? s[rz_new] / b : 0.0;
  p[t] = z[t] + beta * p[t];
}

__global__ void k_sub_mean(int64_t n, double* __restrict__ x, const double* __restrict__ sum) {
  const int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (t < n) x[t] -= sum[0] / (double)n;
}

}  // namespace

// ---------------------------------------------------------------- solver
struct MgLevel {
  Lv L;
  double* w = nullptr;    // 3V conductances
  double* phi = nullptr;  // V
  double* f = nullptr;    // V
  double* r = nullptr;    // V
  bool rb = true;         // red-black Gauss-Seidel (every extent even), else Jacobi
  bool agg = false;       // transfer to the next level by aggregation, else geometric
};

constexpr double kAggAlpha = 1.6;  // over-correction of the aggregated coarse correction

struct MgSolver {
  memd_ctx* c = nullptr;
  std::vector<MgLevel> lv;
  double *x = nullptr, *res = nullptr, *z = nullptr, *p = nullptr, *q = nullptr, *sc = nullptr;
  double* part = nullptr;
  cudaGraphExec_t it_graph = nullptr;
  std::vector<void*> blocks;

  double* alloc(size_t n) {
    void* ptr = memd_dalloc(c, n * sizeof(double));
    if (ptr) blocks.push_back(ptr);
    return (double*)ptr;
  }
  void release() {
    if (it_graph) cudaGraphExecDestroy(it_graph);
    it_graph = nullptr;
    for (void* b : blocks) memd_dfree(c, b);
    blocks.clear();
  }

  void smooth(int l, bool forward, cudaStream_t st) {
    MgLevel& a = lv[l];
    if (a.rb) {
      const int64_t half = a.L.V / 2;
      const int first = forward ? 0 : 1;
      k_rbgs<<<nblk(half), kT, 0, st>>>(a.L, a.w, a.phi, a.f, first);
      k_rbgs<<<nblk(half), kT, 0, st>>>(a.L, a.w, a.phi, a.f, first ^ 1);
    } else {
      k_jacobi_res<<<nblk(a.L.V), kT, 0, st>>>(a.L, a.w, a.phi, a.f, a.r);
      k_jacobi_upd<<<nblk(a.L.V), kT, 0, st>>>(a.L.V, a.phi, a.r, 0.8);
    }
  }

  // z ~ L^-1 f on level l (phi of level l starts at 0); symmetric
  void vcycle(int l, cudaStream_t st) {
    MgLevel& a = lv[l];
    cudaMemsetAsync(a.phi, 0, a.L.V * sizeof(double), st);
    if (l + 1 == (int)lv.size()) {
      const int sweeps = a.L.V <= 512 ? 8 : 12;
      if (a.L.V <= kCoarseSmem) {
        k_coarse_solve<<<1, 1024, 6 * a.L.V * sizeof(double), st>>>(a.L, a.w, a.f, a.phi, sweeps,
                                                                   a.rb ? 1 : 0);
        return;
      }
      for (int s = 0; s < sweeps; ++s) smooth(l, true, st);
      for (int s = 0; s < sweeps; ++s) smooth(l, false, st);
      return;
    }
    MgLevel& b = lv[l + 1];
    smooth(l, true, st);
    smooth(l, true, st);
    k_residual<<<nblk(a.L.V), kT, 0, st>>>(a.L, a.w, a.phi, a.f, a.r);
    if (a.agg)
      k_agg_restrict<<<nblk(b.L.V), kT, 0, st>>>(a.L, b.L, a.r, b.f);
    else
      k_restrict<<<nblk(b.L.V), kT, 0, st>>>(a.L, b.L, a.r, b.f);
    vcycle(l + 1, st);
    if (a.agg)
      k_agg_prolong<<<nblk(a.L.V), kT, 0, st>>>(a.L, b.L, b.phi, kAggAlpha, a.phi);
    else
      k_prolong<<<nblk(a.L.V), kT, 0, st>>>(a.L, b.L, b.phi, a.phi);
    smooth(l, false, st);
    smooth(l, false, st);
  }

  bool build(memd_ctx* ctx, cudaStream_t st) {
    c = ctx;
    const Mesh& m = c->mesh;
    Lv L{m.n[0], m.n[1], m.n[2], m.V};
    const double inv_a2 = 1.0 / (m.a * m.a);
    for (int l = 0;; ++l) {
      MgLevel a;
      a.L = L;
      a.w = alloc(3 * L.V);
      a.phi = alloc(L.V);
      a.f = alloc(L.V);
      a.r = alloc(L.V);
      if (!a.w || !a.phi || !a.f || !a.r) return false;
      a.rb = (L.n0 % 2 == 0) && (L.n1 % 2 == 0) && (L.n2 % 2 == 0);
      if (l == 0)
        k_fine_w<<<nblk(3 * L.V), kT, 0, st>>>(3 * L.V, c->ie64, inv_a2, a.w);
      else if (lv.back().agg)
        k_agg_coarsen<<<nblk(3 * L.V), kT, 0, st>>>(lv.back().L, L, lv.back().w, a.w);
      else
        k_coarsen<<<nblk(3 * L.V), kT, 0, st>>>(lv.back().L, L, lv.back().w, a.w);
      a.agg = !a.rb;  // the way down from this level
      lv.push_back(a);
      if (L.n0 < 4 || L.n1 < 4 || L.n2 < 4 || L.V <= 64) break;
      L.n0 /= 2;
      L.n1 /= 2;
      L.n2 /= 2;
      L.V = (int64_t)L.n0 * L.n1 * L.n2;
    }
    const int64_t V = m.V;
    x = alloc(V);
    res = alloc(V);
    z = alloc(V);
    p = alloc(V);
    q = alloc(V);
    sc = alloc(16);
    part = alloc(reduce_blocks());
    return x && res && z && p && q && sc && part && cudaGetLastError() == cudaSuccess;
  }

  // two CG iterations (the r.z slots alternate), preconditioned by a V-cycle
  void iterations(cudaStream_t st) {
    const int64_t V = lv[0].L.V;
    for (int h = 0; h < 2; ++h) {
      const int old_s = 1 + h, new_s = 2 - h;
      k_apply<<<nblk(V), kT, 0, st>>>(lv[0].L, lv[0].w, p, q);
      launch_dot(p, q, V, part, st);
      launch_finish(part, 0, sc + 0, st);
      k_cg_xr<<<nblk(V), kT, 0, st>>>(V, x, res, p, q, sc, old_s);
      cudaMemcpyAsync(lv[0].f, res, V * sizeof(double), cudaMemcpyDeviceToDevice, st);
      vcycle(0, st);
      cudaMemcpyAsync(z, lv[0].phi, V * sizeof(double), cudaMemcpyDeviceToDevice, st);
      launch_dot(res, z, V, part, st);
      launch_finish(part, 0, sc + new_s, st);
      k_cg_p<<<nblk(V), kT, 0, st>>>(V, p, z, sc, new_s, old_s);
    }
    launch_dot(res, res, V, part, st);
    launch_finish(part, 0, sc + 3, st);
  }

  // A solve in stages, so that one host thread can interleave several
  // solvers on their own streams: begin (to the first residual), then
  // launch_step / check until done, then finish.
  double f2 = 0.0, least = 0.0;
  int its = 0, cap = 0;
  bool done = false;

  memd_status begin(const double* f, int maxit, cudaStream_t st) {
    const int64_t V = lv[0].L.V;
    // r = f - mean(f), x = 0, z = M r, p = z
    cudaMemcpyAsync(res, f, V * sizeof(double), cudaMemcpyDeviceToDevice, st);
    launch_dot(res, nullptr, V, part, st);
    launch_finish(part, 0, sc + 4, st);
    k_sub_mean<<<nblk(V), kT, 0, st>>>(V, res, sc + 4);
    launch_dot(res, res, V, part, st);
    launch_finish(part, 0, sc + 5, st);
    cudaMemsetAsync(x, 0, V * sizeof(double), st);
    cudaMemcpyAsync(lv[0].f, res, V * sizeof(double), cudaMemcpyDeviceToDevice, st);
    vcycle(0, st);
    cudaMemcpyAsync(z, lv[0].phi, V * sizeof(double), cudaMemcpyDeviceToDevice, st);
    cudaMemcpyAsync(p, z, V * sizeof(double), cudaMemcpyDeviceToDevice, st);
    launch_dot(res, z, V, part, st);
    launch_finish(part, 0, sc + 1, st);
    if (!it_graph && c->use_graphs) {
      cudaGraph_t g = nullptr;
      if (cudaStreamBeginCapture(st, cudaStreamCaptureModeThreadLocal) == cudaSuccess) {
        iterations(st);
        if (cudaStreamEndCapture(st, &g) != cudaSuccess ||
            cudaGraphInstantiate(&it_graph, g, 0) != cudaSuccess)
          it_graph = nullptr;
        if (g) cudaGraphDestroy(g);
      }
      cudaGetLastError();
    }
    double h = 0.0;
    if (cudaMemcpyAsync(&h, sc + 5, sizeof(double), cudaMemcpyDeviceToHost, st) != cudaSuccess ||
        cudaStreamSynchronize(st) != cudaSuccess)
      return MEMD_ERR_CUDA;
    f2 = h;
    its = 0;
    done = f2 == 0.0;
    least = f2;
    cap = maxit < 400 ? maxit : 400;
    return MEMD_OK;
  }
  bool running() const { return !done && its < cap; }
  // two iterations queued on st
  memd_status launch_step(cudaStream_t st) {
    if (it_graph) {
      if (cudaGraphLaunch(it_graph, st) != cudaSuccess) return MEMD_ERR_CUDA;
    } else {
      iterations(st);
    }
    its += 2;
    return MEMD_OK;
  }
  // waits for st and tests the residual of the last step
  memd_status check(double tol, cudaStream_t st) {
    double h = 0.0;
    if (cudaMemcpyAsync(&h, sc + 3, sizeof(double), cudaMemcpyDeviceToHost, st) != cudaSuccess ||
        cudaStreamSynchronize(st) != cudaSuccess)
      return MEMD_ERR_CUDA;
    done = h <= tol * tol * f2;
    if (!done && h > 100.0 * least && least <= 1e4 * tol * tol * f2) done = true;
    least = std::min(least, h);
    return MEMD_OK;
  }
  memd_status finish(double* out, int* iters, cudaStream_t st) {
    const int64_t V = lv[0].L.V;
    if (iters) *iters = its;
    // zero-mean solution
    launch_dot(x, nullptr, V, part, st);
    launch_finish(part, 0, sc + 6, st);
    k_sub_mean<<<nblk(V), kT, 0, st>>>(V, x, sc + 6);
    cudaMemcpyAsync(out, x, V * sizeof(double), cudaMemcpyDeviceToDevice, st);
    if (cudaGetLastError() != cudaSuccess) return MEMD_ERR_CUDA;
    return done ? MEMD_OK : MEMD_ERR_RELAX_NOCONV;
  }

  // x = L^-1 f (f of zero mean up to rounding; x of zero mean); stops when
  // |r| <= tol |f| (2-norms), or, once the recursion has reached its
  // rounding floor and the residual grows again (to 100 times its least
  // value), when that least value was below 100 tol |f|; at most
  // min(maxit, 400) iterations
  memd_status solve(const double* f, double* out, double tol, int maxit, int* iters,
                    cudaStream_t st) {
    memd_status s = begin(f, maxit, st);
    while (s == MEMD_OK && running()) {
      s = launch_step(st);
      if (s == MEMD_OK) s = check(tol, st);
    }
    return s == MEMD_OK ? finish(out, iters, st) : s;
  }
};

// ------------------------------------------------------------ entry points
// Cell problems: psi_d (3V, stored), and eps_eff[e][d] = mean over links of
// eps_e (delta_ed - grad_e psi_d) (row e, column d).
// Set on a thread (the request server's admission workers, several of which
// already set systems up at once): that thread's cell problems are solved in
// turn, with one solver's scratch.
namespace {
thread_local bool t_cells_in_turn = false;
}
void memd_mg_cells_in_turn(bool on) { t_cells_in_turn = on; }

memd_status mg_eps_eff(memd_ctx* c, double* psi, double eps_eff[9], double tol, int maxit) {
  const Mesh& m = c->mesh;
  const Lv L{m.n[0], m.n[1], m.n[2], m.V};
  // The three cell problems are independent: each gets its own solver (and
  // scratch) and stream, and this thread interleaves them (each one's two
  // iterations queued, then each one's residual read), so that their small
  // multigrid launches run at once; the results are those of solving them
  // in turn, which a thread set by memd_mg_cells_in_turn does, with one
  // solver on the context's stream.
  const int ns = t_cells_in_turn ? 1 : 3;
  MgSolver S[3];
  double* f[3] = {nullptr, nullptr, nullptr};
  double* U[3] = {nullptr, nullptr, nullptr};
  cudaStream_t sts[3] = {c->stream, nullptr, nullptr};
  cudaEvent_t ready = nullptr;
  memd_status s = MEMD_OK;
  auto cleanup = [&]() {
    // no scratch is released while a stream may still use it
    for (int k = 0; k < 3; ++k)
      if (sts[k]) cudaStreamSynchronize(sts[k]);
    for (MgSolver& x : S) x.release();
    for (int k = 1; k < 3; ++k)
      if (sts[k]) cudaStreamDestroy(sts[k]);
    if (ready) cudaEventDestroy(ready);
  };
  for (int k = 1; k < ns && s == MEMD_OK; ++k)
    if (cudaStreamCreateWithFlags(&sts[k], cudaStreamNonBlocking) != cudaSuccess)
      s = MEMD_ERR_CUDA;
  if (s == MEMD_OK && ns > 1 &&
      (cudaEventCreateWithFlags(&ready, cudaEventDisableTiming) != cudaSuccess ||
       cudaEventRecord(ready, c->stream) != cudaSuccess))
    s = MEMD_ERR_CUDA;
  for (int k = 0; k < ns && s == MEMD_OK; ++k) {
    // the solver's level weights come from 1/eps, written on the context's stream
    if (k > 0 && cudaStreamWaitEvent(sts[k], ready, 0) != cudaSuccess) s = MEMD_ERR_CUDA;
    if (s == MEMD_OK && !S[k].build(c, sts[k])) s = MEMD_ERR_OOM;
    if (s == MEMD_OK) {
      f[k] = S[k].alloc(m.V);
      U[k] = S[k].alloc(3 * m.V);
      if (!f[k] || !U[k]) s = MEMD_ERR_OOM;
    }
  }
  // cell problems d0 .. d0 + ns - 1, problem d0 + k with solver k
  auto solve_cells = [&](int d0) -> memd_status {
    memd_status r = MEMD_OK;
    for (int k = 0; k < ns && r == MEMD_OK; ++k) {
      k_div_eps_unit<<<nblk(m.V), kT, 0, sts[k]>>>(L, c->ie64, d0 + k, 1.0 / m.a, f[k]);
      r = S[k].begin(f[k], maxit, sts[k]);
    }
    bool any = true;
    while (r == MEMD_OK && any) {
      any = false;
      for (int k = 0; k < ns && r == MEMD_OK; ++k)
        if (S[k].running()) r = S[k].launch_step(sts[k]);
      for (int k = 0; k < ns && r == MEMD_OK; ++k)
        if (S[k].running()) {
          r = S[k].check(tol, sts[k]);
          any = true;
        }
    }
    for (int k = 0; k < ns && r == MEMD_OK; ++k) {
      const int d = d0 + k;
      const cudaStream_t st = sts[k];
      r = S[k].finish(psi + d * m.V, nullptr, st);
      if (r != MEMD_OK) break;
      k_flux<<<nblk(3 * m.V), kT, 0, st>>>(L, c->ie64, psi + d * m.V, d, 1.0, 1.0 / m.a, U[k],
                                           0, 1.0);
      for (int e = 0; e < 3; ++e) {
        launch_dot(U[k] + e * m.V, nullptr, m.V, S[k].part, st);
        launch_finish(S[k].part, 0, S[k].sc + 8 + e, st);
      }
      double h[3];
      if (cudaMemcpyAsync(h, S[k].sc + 8, 3 * sizeof(double), cudaMemcpyDeviceToHost, st) !=
              cudaSuccess ||
          cudaStreamSynchronize(st) != cudaSuccess) {
        r = MEMD_ERR_CUDA;
        break;
      }
      for (int e = 0; e < 3; ++e) eps_eff[3 * e + d] = h[e] / (double)m.V;
    }
    return r;
  };
  for (int d0 = 0; d0 < 3 && s == MEMD_OK; d0 += ns) s = solve_cells(d0);
  cleanup();
  return s;
}

// D64 (div D = rho, mean M) -> the relaxed field with the same divergence
// and mean: D = -eps grad phi + sum_d E0_d eps (e_d - grad psi_d),
// L phi = div D64, E0 = eps_eff^-1 (M - mean(-eps grad phi)).
memd_status mg_relax(memd_ctx* c, double* D64, const double* psi, const double eps_eff_inv[9],
                     double tol, int maxit, int* iters) {
  const Mesh& m = c->mesh;
  const cudaStream_t st = c->stream;
  const Lv L{m.n[0], m.n[1], m.n[2], m.V};
  MgSolver S;
  if (!S.build(c, st)) {
    S.release();
    return MEMD_ERR_OOM;
  }
  double* f = S.alloc(m.V);
  double* phi = S.alloc(m.V);
  if (!f || !phi) {
    S.release();
    return MEMD_ERR_OOM;
  }
  // mean of D64 per component
  for (int e = 0; e < 3; ++e) {
    launch_dot(D64 + e * m.V, nullptr, m.V, S.part, st);
    launch_finish(S.part, 0, S.sc + 8 + e, st);
  }
  k_div_links<<<nblk(m.V), kT, 0, st>>>(L, D64, 1.0 / m.a, f);
  memd_status s = S.solve(f, phi, tol, maxit, iters, st);
  if (s == MEMD_OK) {
    // D64 <- -eps grad phi, its mean
    k_flux<<<nblk(3 * m.V), kT, 0, st>>>(L, c->ie64, phi, -1, 0.0, 1.0 / m.a, D64, 0, 1.0);
    for (int e = 0; e < 3; ++e) {
      launch_dot(D64 + e * m.V, nullptr, m.V, S.part, st);
      launch_finish(S.part, 0, S.sc + 11 + e, st);
    }
    double h[6];
    if (cudaMemcpyAsync(h, S.sc + 8, 6 * sizeof(double), cudaMemcpyDeviceToHost, st) !=
            cudaSuccess ||
        cudaStreamSynchronize(st) != cudaSuccess) {
      s = MEMD_ERR_CUDA;
    } else {
      double dm[3], E0[3];
      for (int e = 0; e < 3; ++e) dm[e] = (h[e] - h[3 + e]) / (double)m.V;
      for (int e = 0; e < 3; ++e)
        E0[e] = eps_eff_inv[3 * e] * dm[0] + eps_eff_inv[3 * e + 1] * dm[1] +
                eps_eff_inv[3 * e + 2] * dm[2];
      for (int d = 0; d < 3; ++d)
        if (E0[d] != 0.0)
          k_flux<<<nblk(3 * m.V), kT, 0, st>>>(L, c->ie64, psi + d * m.V, d, 1.0, 1.0 / m.a, D64,
                                               1, E0[d]);
      if (cudaGetLastError() != cudaSuccess) s = MEMD_ERR_CUDA;
    }
  }
  S.release();
  return s;
}

}  // namespace memd
