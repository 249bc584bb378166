// memd_field.cu -- lattice field kernels of MEMD on sm_103a.
//
//   curl_B : plaquette update of Eq. 21 (Faraday), B -= (dt/a) circ(D/eps)
//   curl_D : link update of Eq. 20 (Ampere) without the current,
//            D += (c^2 dt/a) (transpose circulation of B)
//   FP64 circulation / transpose maps used by the relaxation (Sec. II)
//   field energy and Gauss-law diagnostics
//
// The field kernels stream every link each step and are bound by HBM
// bandwidth: x is the fastest index, a warp covers 32 consecutive x, the
// +/-1 neighbours in y and z are rows that the same or adjacent CTAs read,
// so they come from L1/L2.
#include "memd_internal.cuh"
#include "memd_site.cuh"

namespace memd {

namespace {

constexpr int kBX = 32;
constexpr int kBY = 8;
constexpr int kRedThreads = 256;
constexpr int kRedBlocks = 2 * 152;

inline dim3 field_grid(const Mesh& m) {
  return dim3((m.n[0] + kBX - 1) / kBX, (m.n[1] + kBY - 1) / kBY, m.n[2]);
}

template <typename T>
__global__ void __launch_bounds__(kBX* kBY)
    k_curl_B(Mesh m, T* __restrict__ B, const T* __restrict__ D, const T* __restrict__ ie,
             T coef) {
  const int i = blockIdx.x * kBX + threadIdx.x;
  const int j = blockIdx.y * kBY + threadIdx.y;
  const int k = blockIdx.z;
  if (i >= m.n[0] || j >= m.n[1]) return;
  const int64_t V = m.V;
  const int ip = (i + 1 == m.n[0]) ? 0 : i + 1;
  const int jp = (j + 1 == m.n[1]) ? 0 : j + 1;
  const int kp = (k + 1 == m.n[2]) ? 0 : k + 1;
  const int64_t v = vindex(m, i, j, k);
  const int64_t vx = vindex(m, ip, j, k), vy = vindex(m, i, jp, k), vz = vindex(m, i, j, kp);
  const T* Dx = D;
  const T* Dy = D + V;
  const T* Dz = D + 2 * V;
  const T* ix = ie;
  const T* iy = ie + V;
  const T* iz = ie + 2 * V;
  const T Ex = Dx[v] * ix[v], Ey = Dy[v] * iy[v], Ez = Dz[v] * iz[v];
  const T Ey_x = Dy[vx] * iy[vx], Ez_x = Dz[vx] * iz[vx];
  const T Ex_y = Dx[vy] * ix[vy], Ez_y = Dz[vy] * iz[vy];
  const T Ex_z = Dx[vz] * ix[vz], Ey_z = Dy[vz] * iy[vz];
  // circulations: normal x spans (y, z), normal y spans (z, x), normal z spans (x, y)
  B[v] = B[v] - coef * (((Ey + Ez_y) - Ey_z) - Ez);
  B[V + v] = B[V + v] - coef * (((Ez + Ex_z) - Ez_x) - Ex);
  B[2 * V + v] = B[2 * V + v] - coef * (((Ex + Ey_x) - Ex_y) - Ey);
}

template <typename T>
__global__ void __launch_bounds__(kBX* kBY)
    k_curl_D(Mesh m, T* __restrict__ D, const T* __restrict__ B, T coef) {
  const int i = blockIdx.x * kBX + threadIdx.x;
  const int j = blockIdx.y * kBY + threadIdx.y;
  const int k = blockIdx.z;
  if (i >= m.n[0] || j >= m.n[1]) return;
  const int64_t V = m.V;
  const int im = (i == 0) ? m.n[0] - 1 : i - 1;
  const int jm = (j == 0) ? m.n[1] - 1 : j - 1;
  const int km = (k == 0) ? m.n[2] - 1 : k - 1;
  const int64_t v = vindex(m, i, j, k);
  const int64_t vx = vindex(m, im, j, k), vy = vindex(m, i, jm, k), vz = vindex(m, i, j, km);
  const T* Bx = B;
  const T* By = B + V;
  const T* Bz = B + 2 * V;
  const T bx = Bx[v], by = By[v], bz = Bz[v];
  D[v] = D[v] + coef * (((bz - Bz[vy]) - by) + By[vz]);
  D[V + v] = D[V + v] + coef * (((bx - Bx[vz]) - bz) + Bz[vx]);
  D[2 * V + v] = D[2 * V + v] + coef * (((by - By[vx]) - bx) + Bx[vy]);
}

// w = sign * circulation of (ie * u) around every plaquette (FP64)
__global__ void __launch_bounds__(kBX* kBY)
    k_circ64(Mesh m, double* __restrict__ w, const double* __restrict__ u,
             const double* __restrict__ ie, double sign) {
  const int i = blockIdx.x * kBX + threadIdx.x;
  const int j = blockIdx.y * kBY + threadIdx.y;
  const int k = blockIdx.z;
  if (i >= m.n[0] || j >= m.n[1]) return;
  const int64_t V = m.V;
  const int ip = (i + 1 == m.n[0]) ? 0 : i + 1;
  const int jp = (j + 1 == m.n[1]) ? 0 : j + 1;
  const int kp = (k + 1 == m.n[2]) ? 0 : k + 1;
  const int64_t v = vindex(m, i, j, k);
  const int64_t vx = vindex(m, ip, j, k), vy = vindex(m, i, jp, k), vz = vindex(m, i, j, kp);
  const double Ex = u[v] * ie[v], Ey = u[V + v] * ie[V + v], Ez = u[2 * V + v] * ie[2 * V + v];
  const double Ey_x = u[V + vx] * ie[V + vx], Ez_x = u[2 * V + vx] * ie[2 * V + vx];
  const double Ex_y = u[vy] * ie[vy], Ez_y = u[2 * V + vy] * ie[2 * V + vy];
  const double Ex_z = u[vz] * ie[vz], Ey_z = u[V + vz] * ie[V + vz];
  w[v] = sign * (((Ey + Ez_y) - Ey_z) - Ez);
  w[V + v] = sign * (((Ez + Ex_z) - Ez_x) - Ex);
  w[2 * V + v] = sign * (((Ex + Ey_x) - Ex_y) - Ey);
}

// u = transpose of the circulation map applied to the plaquette field p
__global__ void __launch_bounds__(kBX* kBY)
    k_curlT64(Mesh m, double* __restrict__ u, const double* __restrict__ p) {
  const int i = blockIdx.x * kBX + threadIdx.x;
  const int j = blockIdx.y * kBY + threadIdx.y;
  const int k = blockIdx.z;
  if (i >= m.n[0] || j >= m.n[1]) return;
  const int64_t V = m.V;
  const int im = (i == 0) ? m.n[0] - 1 : i - 1;
  const int jm = (j == 0) ? m.n[1] - 1 : j - 1;
  const int km = (k == 0) ? m.n[2] - 1 : k - 1;
  const int64_t v = vindex(m, i, j, k);
  const int64_t vx = vindex(m, im, j, k), vy = vindex(m, i, jm, k), vz = vindex(m, i, j, km);
  const double px = p[v], py = p[V + v], pz = p[2 * V + v];
  u[v] = ((pz - p[2 * V + vy]) - py) + p[V + vz];
  u[V + v] = ((px - p[vz]) - pz) + p[2 * V + vx];
  u[2 * V + v] = ((py - p[V + vx]) - px) + p[vy];
}

__global__ void __launch_bounds__(kBX* kBY)
    k_plaquette_diag(Mesh m, double* __restrict__ diag, const double* __restrict__ ie) {
  const int i = blockIdx.x * kBX + threadIdx.x;
  const int j = blockIdx.y * kBY + threadIdx.y;
  const int k = blockIdx.z;
  if (i >= m.n[0] || j >= m.n[1]) return;
  const int64_t V = m.V;
  const int ip = (i + 1 == m.n[0]) ? 0 : i + 1;
  const int jp = (j + 1 == m.n[1]) ? 0 : j + 1;
  const int kp = (k + 1 == m.n[2]) ? 0 : k + 1;
  const int64_t v = vindex(m, i, j, k);
  const int64_t vx = vindex(m, ip, j, k), vy = vindex(m, i, jp, k), vz = vindex(m, i, j, kp);
  diag[v] = ie[V + v] + ie[2 * V + vy] + ie[V + vz] + ie[2 * V + v];
  diag[V + v] = ie[2 * V + v] + ie[vz] + ie[2 * V + vx] + ie[v];
  diag[2 * V + v] = ie[v] + ie[V + vx] + ie[vy] + ie[V + v];
}

// ------------------------------------------------------------------
// Fused leapfrog field update of one step (Eqs. 20 and 21 without the
// current): B' = B - cB circ(D ie) on every plaquette, then
// D' = D + cD (transpose circulation of B') on every link.
//
// Each CTA owns a TX x TY column tile and marches up a chunk of z planes.
// Shared memory holds E = D ie of planes k, k+1, k+2 (a ring of three) and
// B' of planes k-1, k, each with a one-site halo on the low x / y sides
// (B' there is recomputed rather than exchanged between CTAs).  While plane
// k is computed, the loads for plane k+1 (B, D) and k+2 (D, 1/eps) are
// already in flight in registers, so DRAM latency overlaps the arithmetic.
// D and B are double-buffered (read *_in, write *_out) because neighbouring
// CTAs read the halo of the input.  DRAM traffic per site: D, 1/eps, B read
// once, D', B' written once (60 B in FP32, 120 B in FP64).
template <typename T, int TX, int TY>
__device__ __forceinline__ void fused_tile(const Mesh& m, const T* __restrict__ Din,
                                           const T* __restrict__ Bin, const T* __restrict__ ie,
                                           T* __restrict__ Dout, T* __restrict__ Bout, T cB, T cD,
                                           int tile_x, int tile_y, int tile_z, int zchunk) {
  constexpr int EX = TX + 2, EY = TY + 2, BX = TX + 1, BY = TY + 1;
  constexpr int NT = TX * TY;
  constexpr int NE = (EX * EY + NT - 1) / NT;  // E-region elements per thread
  constexpr int NB = (BX * BY + NT - 1) / NT;  // B-region elements per thread
  __shared__ T sE[3][3][EY][EX];
  __shared__ T sB[2][3][BY][BX];
  const int nx = m.n[0], ny = m.n[1], nz = m.n[2];
  const int64_t V = m.V;
  const int64_t P = (int64_t)nx * ny;
  const int x0 = tile_x * TX, y0 = tile_y * TY;
  const int z0 = tile_z * zchunk;
  const int z1 = min(z0 + zchunk, nz);
  const int tid = threadIdx.y * TX + threadIdx.x;

  // in-plane offsets of this thread's E- and B-region elements (periodic)
  int eo[NE], bo[NB];
  bool bin_[NB];
#pragma unroll
  for (int j = 0; j < NE; ++j) {
    int e = tid + j * NT;
    if (e >= EX * EY) e = EX * EY - 1;
    const int ey = e / EX, ex = e - ey * EX;
    int x = x0 - 1 + ex, y = y0 - 1 + ey;
    x = (x < 0) ? x + nx : (x >= nx ? x - nx : x);
    y = (y < 0) ? y + ny : (y >= ny ? y - ny : y);
    if (x >= nx) x = nx - 1;  // only when the tile is wider than the mesh (unused)
    if (y >= ny) y = ny - 1;
    eo[j] = y * nx + x;
  }
#pragma unroll
  for (int j = 0; j < NB; ++j) {
    int e = tid + j * NT;
    const bool real = e < BX * BY;
    if (!real) e = BX * BY - 1;
    const int by = e / BX, bx = e - by * BX;
    int x = x0 - 1 + bx, y = y0 - 1 + by;
    bin_[j] = real && bx >= 1 && by >= 1 && x < nx && y < ny;
    x = (x < 0) ? x + nx : (x >= nx ? x - nx : x);
    y = (y < 0) ? y + ny : (y >= ny ? y - ny : y);
    if (x >= nx) x = nx - 1;
    if (y >= ny) y = ny - 1;
    bo[j] = y * nx + x;
  }
  const int tx = threadIdx.x, ty = threadIdx.y;
  const bool mine = (x0 + tx < nx) && (y0 + ty < ny);
  const int io = min(y0 + ty, ny - 1) * nx + min(x0 + tx, nx - 1);

  auto plane = [&](int k) -> int64_t { return (int64_t)k * P; };
  auto wrapz = [&](int k) -> int { return k >= nz ? k - nz : (k < 0 ? k + nz : k); };

  // registers: D and 1/eps for an E plane, B for a B plane, D of the own site
  T rD[NE][3], rI[NE][3], rB[NB][3], rDs[3];
  auto fetch_E = [&](int k) {
    const int64_t pk = plane(k);
#pragma unroll
    for (int j = 0; j < NE; ++j)
#pragma unroll
      for (int c = 0; c < 3; ++c) {
        rD[j][c] = Din[c * V + pk + eo[j]];
        rI[j][c] = ie[c * V + pk + eo[j]];
      }
  };
  auto store_E = [&](int slot) {
#pragma unroll
    for (int j = 0; j < NE; ++j) {
      const int e = tid + j * NT;
      if (e < EX * EY) {
        const int ey = e / EX, ex = e - ey * EX;
#pragma unroll
        for (int c = 0; c < 3; ++c) sE[slot][c][ey][ex] = rD[j][c] * rI[j][c];
      }
    }
  };
  auto fetch_B = [&](int k, T (&dst)[NB][3]) {
    const int64_t pk = plane(k);
#pragma unroll
    for (int j = 0; j < NB; ++j)
#pragma unroll
      for (int c = 0; c < 3; ++c) dst[j][c] = Bin[c * V + pk + bo[j]];
  };
  auto fetch_Ds = [&](int k, T (&dst)[3]) {
    const int64_t pk = plane(k);
#pragma unroll
    for (int c = 0; c < 3; ++c) dst[c] = Din[c * V + pk + io];
  };
  // B' of plane k on the tile and its low halo, from E in slots ec (k) and
  // en (k+1) and B of plane k in registers; interior values also to Bout
  auto compute_B = [&](int k, int ec, int en, int slot, const T (&bb)[NB][3], bool store) {
    const int64_t pk = plane(k);
#pragma unroll
    for (int j = 0; j < NB; ++j) {
      const int e = tid + j * NT;
      if (e < BX * BY) {
        const int by = e / BX, bx = e - by * BX;
        const T Ex = sE[ec][0][by][bx], Ey = sE[ec][1][by][bx], Ez = sE[ec][2][by][bx];
        const T Ey_x = sE[ec][1][by][bx + 1], Ez_x = sE[ec][2][by][bx + 1];
        const T Ex_y = sE[ec][0][by + 1][bx], Ez_y = sE[ec][2][by + 1][bx];
        const T Ex_z = sE[en][0][by][bx], Ey_z = sE[en][1][by][bx];
        const T bxv = bb[j][0] - cB * (((Ey + Ez_y) - Ey_z) - Ez);
        const T byv = bb[j][1] - cB * (((Ez + Ex_z) - Ez_x) - Ex);
        const T bzv = bb[j][2] - cB * (((Ex + Ey_x) - Ex_y) - Ey);
        sB[slot][0][by][bx] = bxv;
        sB[slot][1][by][bx] = byv;
        sB[slot][2][by][bx] = bzv;
        if (store && bin_[j]) {
          Bout[pk + bo[j]] = bxv;
          Bout[V + pk + bo[j]] = byv;
          Bout[2 * V + pk + bo[j]] = bzv;
        }
      }
    }
  };

  // prologue: E of z0-1, z0, z0+1 and B' of z0-1 (recomputed halo plane)
  {
    T bb[NB][3];
    fetch_E(wrapz(z0 - 1));
    fetch_B(wrapz(z0 - 1), bb);
    store_E(0);
    fetch_E(z0);
    store_E(1);
    fetch_E(wrapz(z0 + 1));
    store_E(2);
    __syncthreads();
    compute_B(wrapz(z0 - 1), 0, 1, 0, bb, false);
  }
  T cBr[NB][3], cDs[3];
  fetch_B(z0, cBr);
  fetch_Ds(z0, cDs);
  int ec = 1, en = 2, ef = 0, bp = 0, bc = 1;
  for (int k = z0; k < z1; ++k) {
    const bool more = k + 1 < z1;
    if (more) {  // in flight while plane k is computed
      fetch_E(wrapz(k + 2));
      fetch_B(k + 1, rB);
      fetch_Ds(k + 1, rDs);
    }
    __syncthreads();  // E(k+1) stored, sB[bc] free
    compute_B(k, ec, en, bc, cBr, true);
    __syncthreads();
    if (mine) {
      const int bx = tx + 1, by = ty + 1;
      const int64_t v = plane(k) + io;
      const T Bx = sB[bc][0][by][bx], By = sB[bc][1][by][bx], Bz = sB[bc][2][by][bx];
      Dout[v] = cDs[0] + cD * (((Bz - sB[bc][2][by - 1][bx]) - By) + sB[bp][1][by][bx]);
      Dout[V + v] = cDs[1] + cD * (((Bx - sB[bp][0][by][bx]) - Bz) + sB[bc][2][by][bx - 1]);
      Dout[2 * V + v] = cDs[2] + cD * (((By - sB[bc][1][by][bx - 1]) - Bx) + sB[bc][0][by - 1][bx]);
    }
    if (more) {
      store_E(ef);
#pragma unroll
      for (int j = 0; j < NB; ++j)
#pragma unroll
        for (int c = 0; c < 3; ++c) cBr[j][c] = rB[j][c];
#pragma unroll
      for (int c = 0; c < 3; ++c) cDs[c] = rDs[c];
    }
    const int t = ec;
    ec = en;
    en = ef;
    ef = t;
    bp ^= 1;
    bc ^= 1;
  }
}

template <typename T, int TY, int PF>
__global__ void __launch_bounds__(34 * (TY + 2))
    k_fused_site(Mesh m, const T* __restrict__ Din, const T* __restrict__ Bin,
                 const T* __restrict__ ie, T* __restrict__ Dout, T* __restrict__ Bout, T cB,
                 T cD, int zchunk) {
  site_tile<T, TY, PF>(m, Din, Bin, ie, Dout, Bout, cB, cD, blockIdx.x, blockIdx.y, blockIdx.z,
                       zchunk, threadIdx.x, threadIdx.y, true, CtaSync{});
}

// Many independent systems in one launch: CTA b works on a site tile of
// replica cta_rep[b]; each replica's tiles are a contiguous range of CTAs.
template <typename T, int TY, int PF, int TX>
__global__ void __launch_bounds__((TX + 2) * (TY + 2))
    k_fused_site_batch(const RepDesc* __restrict__ desc, const int* __restrict__ cta_rep, int par) {
  const RepDesc& r = desc[cta_rep[blockIdx.x]];
  const int local = blockIdx.x - r.f_first;
  const int per_z = r.f_tx * r.f_ty;
  const int tz = local / per_z, rem = local - tz * per_z;
  const int ty = rem / r.f_tx, tx = rem - ty * r.f_tx;
  site_tile<T, TY, PF, CtaSync, TX>(r.m, (const T*)r.D[par], (const T*)r.B[par], (const T*)r.ie,
                                    (T*)r.D[par ^ 1], (T*)r.B[par ^ 1], (T)r.sp.coefB,
                                    (T)r.sp.coefD, tx, ty, tz, r.f_zchunk, threadIdx.x,
                                    threadIdx.y, true, CtaSync{});
}

template <typename T, int TX, int TY>
__global__ void __launch_bounds__(TX* TY)
    k_fused_curl(Mesh m, const T* __restrict__ Din, const T* __restrict__ Bin,
                 const T* __restrict__ ie, T* __restrict__ Dout, T* __restrict__ Bout, T cB,
                 T cD, int zchunk) {
  fused_tile<T, TX, TY>(m, Din, Bin, ie, Dout, Bout, cB, cD, blockIdx.x, blockIdx.y, blockIdx.z,
                        zchunk);
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

__device__ inline double block_max(double x, double* sh) {
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

__device__ inline void coords(const Mesh& m, int64_t v, int& i, int& j, int& k) {
  i = (int)(v % m.n[0]);
  const int64_t r = v / m.n[0];
  j = (int)(r % m.n[1]);
  k = (int)(r / m.n[1]);
}

template <typename T>
__global__ void __launch_bounds__(kRedThreads)
    k_field_energy(Mesh m, const T* __restrict__ D, const T* __restrict__ B,
                   const T* __restrict__ ie, double coefB, double* part_el, double* part_mag) {
  __shared__ double sh[kRedThreads / 32];
  const int64_t V = m.V;
  double el = 0.0, mag = 0.0;
  for (int64_t v = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; v < V;
       v += (int64_t)gridDim.x * blockDim.x) {
    int i, j, k;
    coords(m, v, i, j, k);
    const int ip = (i + 1 == m.n[0]) ? 0 : i + 1;
    const int jp = (j + 1 == m.n[1]) ? 0 : j + 1;
    const int kp = (k + 1 == m.n[2]) ? 0 : k + 1;
    const int64_t vx = vindex(m, ip, j, k), vy = vindex(m, i, jp, k), vz = vindex(m, i, j, kp);
    double E[3], Ex_[3], Ey_[3], Ez_[3];
    for (int d = 0; d < 3; ++d) {
      const double dd = (double)D[d * V + v], ii = (double)ie[d * V + v];
      E[d] = dd * ii;
      el += 0.5 * dd * dd * ii;
      Ex_[d] = (double)D[d * V + vx] * (double)ie[d * V + vx];
      Ey_[d] = (double)D[d * V + vy] * (double)ie[d * V + vy];
      Ez_[d] = (double)D[d * V + vz] * (double)ie[d * V + vz];
    }
    const double cx = ((E[1] + Ey_[2]) - Ez_[1]) - E[2];
    const double cy = ((E[2] + Ez_[0]) - Ex_[2]) - E[0];
    const double cz = ((E[0] + Ex_[1]) - Ey_[0]) - E[1];
    const double bx = (double)B[v], by = (double)B[V + v], bz = (double)B[2 * V + v];
    mag += bx * (bx - coefB * cx) + by * (by - coefB * cy) + bz * (bz - coefB * cz);
  }
  const double s1 = block_sum(el, sh);
  const double s2 = block_sum(mag, sh);
  if (threadIdx.x == 0) {
    part_el[blockIdx.x] = s1;
    part_mag[blockIdx.x] = s2;
  }
}

template <typename T>
__global__ void __launch_bounds__(kRedThreads)
    k_gauss_check(Mesh m, const T* __restrict__ D, const long long* __restrict__ Lg,
                  const long long* __restrict__ Q, double a2, double* part_res,
                  unsigned long long* mismatch) {
  __shared__ double sh[kRedThreads / 32];
  const int64_t V = m.V;
  double res = 0.0;
  unsigned long long bad = 0;
  const double unit = 3.552713678800501e-15;  // 2^-48
  for (int64_t v = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; v < V;
       v += (int64_t)gridDim.x * blockDim.x) {
    int i, j, k;
    coords(m, v, i, j, k);
    const int im = (i == 0) ? m.n[0] - 1 : i - 1;
    const int jm = (j == 0) ? m.n[1] - 1 : j - 1;
    const int km = (k == 0) ? m.n[2] - 1 : k - 1;
    const int64_t vx = vindex(m, im, j, k), vy = vindex(m, i, jm, k), vz = vindex(m, i, j, km);
    const long long dl =
        (Lg[kLT * tl_pair(0, v)] - Lg[kLT * tl_pair(0, vx)]) +
        (Lg[kLT * tl_pair(1, v)] - Lg[kLT * tl_pair(1, vy)]) +
        (Lg[kLT * tl_pair(2, v)] - Lg[kLT * tl_pair(2, vz)]);
    if (dl != Q[v]) ++bad;
    const double dd = ((double)D[v] - (double)D[vx]) + ((double)D[V + v] - (double)D[V + vy]) +
                      ((double)D[2 * V + v] - (double)D[2 * V + vz]);
    res = fmax(res, fabs(dd * a2 - (double)Q[v] * unit));
  }
  const double r = block_max(res, sh);
  if (threadIdx.x == 0) part_res[blockIdx.x] = r;
  if (bad) atomicAdd(mismatch, bad);
}

// ---------------------------------------------------------- fused PCG
// Three of the four kernels of one preconditioned-CG iteration on plaquette
// rotations (the fourth is the transpose map k_curlT64).  Every CTA reduces
// the per-CTA partial sums of the previous kernel itself, in the same order,
// so the scalars alpha and beta are identical everywhere without a separate
// reduction launch.  Slots of the scalar array sc follow the host code.
constexpr int kCgDone = 14, kCgTol = 15, kCgEmax = 4;

// all threads of the CTA get op(part[0..n)) (op 0: sum, 1: max), fixed order
__device__ inline double cta_reduce(const double* __restrict__ part, int n, int op, double* sh) {
  double x = 0.0;
  for (int t = threadIdx.x; t < n; t += blockDim.x) x = op ? fmax(x, part[t]) : x + part[t];
  for (int o = 16; o > 0; o >>= 1) {
    const double y = __shfl_down_sync(0xffffffffu, x, o);
    x = op ? fmax(x, y) : x + y;
  }
  if ((threadIdx.x & 31) == 0) sh[threadIdx.x >> 5] = x;
  __syncthreads();
  if (threadIdx.x == 0) {
    double r = 0.0;
    for (int t = 0; t < (int)(blockDim.x >> 5); ++t) r = op ? fmax(r, sh[t]) : r + sh[t];
    sh[32] = r;
  }
  __syncthreads();
  const double r = sh[32];
  __syncthreads();
  return r;
}

// w = circulation of (ie u) on every plaquette, and this CTA's share of p.w
__global__ void __launch_bounds__(kRedThreads)
    k_cg_apply(Mesh m, double* __restrict__ w, const double* __restrict__ u,
               const double* __restrict__ ie, const double* __restrict__ p,
               double* __restrict__ part) {
  __shared__ double sh[kRedThreads / 32];
  const int64_t V = m.V;
  double acc = 0.0;
  for (int64_t v = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; v < V;
       v += (int64_t)gridDim.x * blockDim.x) {
    int i, j, k;
    coords(m, v, i, j, k);
    const int ip = (i + 1 == m.n[0]) ? 0 : i + 1;
    const int jp = (j + 1 == m.n[1]) ? 0 : j + 1;
    const int kp = (k + 1 == m.n[2]) ? 0 : k + 1;
    const int64_t vx = vindex(m, ip, j, k), vy = vindex(m, i, jp, k), vz = vindex(m, i, j, kp);
    const double Ex = u[v] * ie[v], Ey = u[V + v] * ie[V + v], Ez = u[2 * V + v] * ie[2 * V + v];
    const double Ey_x = u[V + vx] * ie[V + vx], Ez_x = u[2 * V + vx] * ie[2 * V + vx];
    const double Ex_y = u[vy] * ie[vy], Ez_y = u[2 * V + vy] * ie[2 * V + vy];
    const double Ex_z = u[vz] * ie[vz], Ey_z = u[V + vz] * ie[V + vz];
    const double wx = ((Ey + Ez_y) - Ey_z) - Ez;
    const double wy = ((Ez + Ex_z) - Ez_x) - Ex;
    const double wz = ((Ex + Ey_x) - Ex_y) - Ey;
    w[v] = wx;
    w[V + v] = wy;
    w[2 * V + v] = wz;
    acc += p[v] * wx + p[V + v] * wy + p[2 * V + v] * wz;
  }
  const double s = block_sum(acc, sh);
  if (threadIdx.x == 0) part[blockIdx.x] = s;
}

// alpha = rz / p.w; D += alpha u; r -= alpha w; z = r / diag; shares of r.z
// and of max |r|.  Frozen (kCgDone) iterations change nothing.
__global__ void __launch_bounds__(kRedThreads)
    k_cg_update(int64_t n, double* __restrict__ D, const double* __restrict__ u,
                double* __restrict__ r, const double* __restrict__ w, double* __restrict__ z,
                const double* __restrict__ diag, const double* __restrict__ part_pw,
                const double* __restrict__ sc, int rz_slot, double* __restrict__ part_rz,
                double* __restrict__ part_rmax) {
  __shared__ double sh[33];
  const double pw = cta_reduce(part_pw, gridDim.x, 0, sh);
  const bool done = sc[kCgDone] != 0.0;
  const double alpha = (!done && pw > 0.0) ? sc[rz_slot] / pw : 0.0;
  double rz = 0.0, mx = 0.0;
  for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < n;
       t += (int64_t)gridDim.x * blockDim.x) {
    double rn = r[t];
    double zn;
    if (!done) {
      D[t] += alpha * u[t];
      rn = rn - alpha * w[t];
      r[t] = rn;
      zn = rn / diag[t];
      z[t] = zn;
    } else {
      zn = z[t];
    }
    rz += rn * zn;
    mx = fmax(mx, fabs(rn));
  }
  const double s1 = block_sum(rz, sh);
  const double s2 = block_max(mx, sh);
  if (threadIdx.x == 0) {
    part_rz[blockIdx.x] = s1;
    part_rmax[blockIdx.x] = s2;
  }
}

// rz_new = r.z, freeze when max|r| <= tol max|E|, else p = z + (rz_new/rz_old) p
__global__ void __launch_bounds__(kRedThreads)
    k_cg_direction(int64_t n, double* __restrict__ p, const double* __restrict__ z,
                   double* __restrict__ sc, const double* __restrict__ part_rz,
                   const double* __restrict__ part_rmax, int nparts, int rz_new, int rz_old) {
  __shared__ double sh[33];
  const double rzn = cta_reduce(part_rz, nparts, 0, sh);
  const double rmax = cta_reduce(part_rmax, nparts, 1, sh);
  if (sc[kCgDone] != 0.0) return;
  if (rmax <= sc[kCgTol] * sc[kCgEmax]) {
    if (blockIdx.x == 0 && threadIdx.x == 0) sc[kCgDone] = 1.0;
    return;
  }
  if (blockIdx.x == 0 && threadIdx.x == 0) sc[rz_new] = rzn;
  const double ro = sc[rz_old];
  const double beta = (ro != 0.0) ? rzn / ro : 0.0;
  for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < n;
       t += (int64_t)gridDim.x * blockDim.x)
    p[t] = z[t] + beta * p[t];
}

}  // namespace

void launch_curl_B(const Mesh& m, int prec, void* B, const void* D, const void* ie,
                   double coef, cudaStream_t st) {
  const dim3 blk(kBX, kBY, 1);
  if (prec == 1)
    k_curl_B<float><<<field_grid(m), blk, 0, st>>>(m, (float*)B, (const float*)D,
                                                   (const float*)ie, (float)coef);
  else
    k_curl_B<double><<<field_grid(m), blk, 0, st>>>(m, (double*)B, (const double*)D,
                                                    (const double*)ie, coef);
}

void launch_curl_D(const Mesh& m, int prec, void* D, const void* B, double coef,
                   cudaStream_t st) {
  const dim3 blk(kBX, kBY, 1);
  if (prec == 1)
    k_curl_D<float><<<field_grid(m), blk, 0, st>>>(m, (float*)D, (const float*)B, (float)coef);
  else
    k_curl_D<double><<<field_grid(m), blk, 0, st>>>(m, (double*)D, (const double*)B, coef);
}

namespace {
template <typename T, int TY>
void fused_launch_t(const Mesh& m, const void* Din, const void* Bin, const void* ie, void* Dout,
                    void* Bout, double cB, double cD, int zchunk, cudaStream_t st) {
  constexpr int TX = 32;
  const dim3 grid((m.n[0] + TX - 1) / TX, (m.n[1] + TY - 1) / TY, (m.n[2] + zchunk - 1) / zchunk);
  k_fused_curl<T, TX, TY><<<grid, dim3(TX, TY, 1), 0, st>>>(
      m, (const T*)Din, (const T*)Bin, (const T*)ie, (T*)Dout, (T*)Bout, (T)cB, (T)cD, zchunk);
}
}  // namespace

namespace {
template <typename T, int TY, int PF>
void site_launch_t(const Mesh& m, const void* Din, const void* Bin, const void* ie, void* Dout,
                   void* Bout, double cB, double cD, int zchunk, cudaStream_t st) {
  const dim3 grid((m.n[0] + 31) / 32, (m.n[1] + TY - 1) / TY, (m.n[2] + zchunk - 1) / zchunk);
  k_fused_site<T, TY, PF><<<grid, dim3(34, TY + 2, 1), 0, st>>>(
      m, (const T*)Din, (const T*)Bin, (const T*)ie, (T*)Dout, (T*)Bout, (T)cB, (T)cD, zchunk);
}
template <typename T, int TY>
void site_launch_pf(int pf, const Mesh& m, const void* Din, const void* Bin, const void* ie,
                    void* Dout, void* Bout, double cB, double cD, int zchunk, cudaStream_t st) {
  if (pf >= 2)
    site_launch_t<T, TY, 2>(m, Din, Bin, ie, Dout, Bout, cB, cD, zchunk, st);
  else
    site_launch_t<T, TY, 1>(m, Din, Bin, ie, Dout, Bout, cB, cD, zchunk, st);
}
}  // namespace

void launch_fused_curl(const Mesh& m, int prec, const void* Din, const void* Bin, const void* ie,
                       void* Dout, void* Bout, double cB, double cD, FusedCfg cfg,
                       cudaStream_t st) {
  if (cfg.zchunk < 1) cfg = fused_default(m);
  if (cfg.zchunk > m.n[2]) cfg.zchunk = m.n[2];
  if (cfg.site) {
    const int pf = cfg.site;
    if (prec == 1) {
      if (cfg.ty == 4)
        site_launch_pf<float, 4>(pf, m, Din, Bin, ie, Dout, Bout, cB, cD, cfg.zchunk, st);
      else if (cfg.ty == 16)
        site_launch_pf<float, 16>(pf, m, Din, Bin, ie, Dout, Bout, cB, cD, cfg.zchunk, st);
      else
        site_launch_pf<float, 8>(pf, m, Din, Bin, ie, Dout, Bout, cB, cD, cfg.zchunk, st);
    } else {
      if (cfg.ty == 4)
        site_launch_pf<double, 4>(pf, m, Din, Bin, ie, Dout, Bout, cB, cD, cfg.zchunk, st);
      else
        site_launch_pf<double, 8>(pf, m, Din, Bin, ie, Dout, Bout, cB, cD, cfg.zchunk, st);
    }
    return;
  }
  if (prec == 1) {
    switch (cfg.ty) {
      case 4: fused_launch_t<float, 4>(m, Din, Bin, ie, Dout, Bout, cB, cD, cfg.zchunk, st); break;
      case 16: fused_launch_t<float, 16>(m, Din, Bin, ie, Dout, Bout, cB, cD, cfg.zchunk, st); break;
      default: fused_launch_t<float, 8>(m, Din, Bin, ie, Dout, Bout, cB, cD, cfg.zchunk, st);
    }
  } else {
    // FP64 tiles stop at 8 rows: 16 would exceed the 48 KB of static shared memory
    if (cfg.ty == 4)
      fused_launch_t<double, 4>(m, Din, Bin, ie, Dout, Bout, cB, cD, cfg.zchunk, st);
    else
      fused_launch_t<double, 8>(m, Din, Bin, ie, Dout, Bout, cB, cD, cfg.zchunk, st);
  }
}

FusedCfg fused_default(const Mesh& m) {
  // enough CTAs to fill the GPU a few times over, but chunks long enough
  // that the recomputed prologue plane stays a small overhead
  FusedCfg c{8, 1, 0, 0, 0};
  const int64_t tiles = (int64_t)((m.n[0] + 31) / 32) * ((m.n[1] + 7) / 8);
  const int64_t target = 4 * 152;
  const int64_t nchunks = (target + tiles - 1) / tiles;
  int64_t zc = (m.n[2] + nchunks - 1) / nchunks;
  if (zc < 4) zc = 4;
  if (zc > m.n[2]) zc = m.n[2];
  c.zchunk = (int)zc;
  return c;
}

namespace {
template <typename T, int TY, int PF>
void batch_launch_t(const RepDesc* desc, const int* cta_rep, int nctas, int par, int tw,
                    cudaStream_t st) {
  if (tw == 16)
    k_fused_site_batch<T, TY, PF, 16><<<nctas, dim3(18, TY + 2, 1), 0, st>>>(desc, cta_rep, par);
  else
    k_fused_site_batch<T, TY, PF, 32><<<nctas, dim3(34, TY + 2, 1), 0, st>>>(desc, cta_rep, par);
}
template <typename T>
void batch_launch_ty(const RepDesc* desc, const int* cta_rep, int nctas, int par, int ty, int pf,
                     int tw, cudaStream_t st) {
  if (ty == 4) {
    if (pf >= 2)
      batch_launch_t<T, 4, 2>(desc, cta_rep, nctas, par, tw, st);
    else
      batch_launch_t<T, 4, 1>(desc, cta_rep, nctas, par, tw, st);
  } else if (ty == 16 && sizeof(T) == 4) {
    if (pf >= 2)
      batch_launch_t<float, 16, 2>(desc, cta_rep, nctas, par, tw, st);
    else
      batch_launch_t<float, 16, 1>(desc, cta_rep, nctas, par, tw, st);
  } else {
    if (pf >= 2)
      batch_launch_t<T, 8, 2>(desc, cta_rep, nctas, par, tw, st);
    else
      batch_launch_t<T, 8, 1>(desc, cta_rep, nctas, par, tw, st);
  }
}
}  // namespace

void launch_fused_batch(int prec, const RepDesc* desc, const int* cta_rep, int nctas, int par,
                        int ty, int pf, int tw, cudaStream_t st) {
  if (nctas <= 0) return;
  if (prec == 1)
    batch_launch_ty<float>(desc, cta_rep, nctas, par, ty, pf, tw, st);
  else
    batch_launch_ty<double>(desc, cta_rep, nctas, par, ty, pf, tw, st);
}

int fused_candidates(const Mesh& m, int prec, FusedCfg* out, int cap) {
  static const int tys[3] = {4, 8, 16};
  static const int zcs[8] = {1, 2, 4, 8, 16, 32, 64, 128};
  int n = 0;
  for (int a = 0; a < (prec == 1 ? 3 : 2); ++a)
    for (int b = 0; b < 8; ++b) {
      if (zcs[b] > m.n[2] && b > 0 && zcs[b - 1] >= m.n[2]) continue;
      if (n < cap) out[n++] = FusedCfg{tys[a], zcs[b] < m.n[2] ? zcs[b] : m.n[2], 0, 0, 0};
    }
  return n;
}

void launch_cg_apply(const Mesh& m, double* w, const double* u, const double* ie,
                     const double* p, double* part, cudaStream_t st) {
  k_cg_apply<<<kRedBlocks, kRedThreads, 0, st>>>(m, w, u, ie, p, part);
}

void launch_cg_update(int64_t n, double* D, const double* u, double* r, const double* w,
                      double* z, const double* diag, const double* part_pw, const double* sc,
                      int rz_slot, double* part_rz, double* part_rmax, cudaStream_t st) {
  k_cg_update<<<kRedBlocks, kRedThreads, 0, st>>>(n, D, u, r, w, z, diag, part_pw, sc, rz_slot,
                                                  part_rz, part_rmax);
}

void launch_cg_direction(int64_t n, double* p, const double* z, double* sc, const double* part_rz,
                         const double* part_rmax, int rz_new, int rz_old, cudaStream_t st) {
  k_cg_direction<<<kRedBlocks, kRedThreads, 0, st>>>(n, p, z, sc, part_rz, part_rmax, kRedBlocks,
                                                     rz_new, rz_old);
}

void launch_circ64(const Mesh& m, double* w, const double* u, const double* ie, double sign,
                   cudaStream_t st) {
  k_circ64<<<field_grid(m), dim3(kBX, kBY, 1), 0, st>>>(m, w, u, ie, sign);
}

void launch_curlT64(const Mesh& m, double* u, const double* p, cudaStream_t st) {
  k_curlT64<<<field_grid(m), dim3(kBX, kBY, 1), 0, st>>>(m, u, p);
}

void launch_plaquette_diag(const Mesh& m, double* diag, const double* ie, cudaStream_t st) {
  k_plaquette_diag<<<field_grid(m), dim3(kBX, kBY, 1), 0, st>>>(m, diag, ie);
}

void launch_field_energy(const Mesh& m, int prec, const void* D, const void* B, const void* ie,
                         double coefB, double* part_el, double* part_mag, cudaStream_t st) {
  if (prec == 1)
    k_field_energy<float><<<kRedBlocks, kRedThreads, 0, st>>>(
        m, (const float*)D, (const float*)B, (const float*)ie, coefB, part_el, part_mag);
  else
    k_field_energy<double><<<kRedBlocks, kRedThreads, 0, st>>>(
        m, (const double*)D, (const double*)B, (const double*)ie, coefB, part_el, part_mag);
}

// block sums over the links of E = D ie: part[b] of E^2 (all 3V links),
// part[(1 + d) R + b] of E_d (the V links of component d)
template <typename T>
__global__ void __launch_bounds__(kRedThreads)
    k_field_moments(const T* __restrict__ D, const T* __restrict__ ie, int64_t V, double* part) {
  __shared__ double sh[kRedThreads / 32];
  const int R = (int)gridDim.x;
  double s2 = 0.0, s[3] = {0.0, 0.0, 0.0};
  for (int64_t v = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; v < V;
       v += (int64_t)gridDim.x * blockDim.x)
    for (int d = 0; d < 3; ++d) {
      const double e = (double)D[d * V + v] * (double)ie[d * V + v];
      s[d] += e;
      s2 += e * e;
    }
  s2 = block_sum(s2, sh);
  if (threadIdx.x == 0) part[blockIdx.x] = s2;
  for (int d = 0; d < 3; ++d) {
    const double t = block_sum(s[d], sh);
    if (threadIdx.x == 0) part[(1 + d) * R + blockIdx.x] = t;
  }
}

void launch_field_moments(int prec, const void* D, const void* ie, int64_t V, double* part,
                          cudaStream_t st) {
  if (prec == 1)
    k_field_moments<float><<<kRedBlocks, kRedThreads, 0, st>>>((const float*)D, (const float*)ie,
                                                              V, part);
  else
    k_field_moments<double><<<kRedBlocks, kRedThreads, 0, st>>>((const double*)D,
                                                               (const double*)ie, V, part);
}

void launch_gauss_check(const Mesh& m, int prec, const void* D, const long long* Lg,
                        const long long* Q, double a2, double* part_res,
                        unsigned long long* mismatch, cudaStream_t st) {
  if (prec == 1)
    k_gauss_check<float><<<kRedBlocks, kRedThreads, 0, st>>>(m, (const float*)D, Lg, Q, a2,
                                                            part_res, mismatch);
  else
    k_gauss_check<double><<<kRedBlocks, kRedThreads, 0, st>>>(m, (const double*)D, Lg, Q, a2,
                                                             part_res, mismatch);
}

}  // namespace memd
