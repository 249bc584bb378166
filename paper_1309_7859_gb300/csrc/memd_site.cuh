// memd_site.cuh -- the one-thread-per-site fused field update (B' from the
// circulation of E = D / eps, then D' from the curl of B', Eq. 20 a-b),
// shared by the field kernels and the single-launch step kernel.
#pragma once
#include "memd_internal.cuh"

namespace memd {

// Fused field update, one thread per site of the tile and of its halo ring.
// A CTA of (TX + 2) x (TY + 2) threads covers the TX x TY tile (TX = 32, or 16
// for narrow meshes) plus one site on every side.  Each thread loads D, 1/eps and B of its own site only (nine
// values a plane, one base pointer), writes its E = D / eps into the shared
// ring of planes k, k+1, k+2, computes B' at its site (tile and low halo),
// and, inside the tile, D' from its own D kept in registers.  Loads run PF
// planes ahead of the plane being computed (register queues), so that about
// 9 PF values per thread are in flight while a plane is computed.  Same
// arithmetic per site as k_fused_curl.
//
// Tp (optional): transfers not yet applied to D (int64 transfer words only,
// component major: tw_index with cmV = V): D(site) is then read as D + Tp
// scale, rounded exactly as their application would (pending_inc).

// (T)((double)t * scale), the increment a transfer t adds to D.  With FP32
// fields and a power-of-two scale (exact32) it is computed as the rounded
// conversion of t to float times the scale, which is the same value (t is
// exact in double, scaling by a power of two is exact, and rounding commutes
// with it) without FP64 arithmetic.
template <typename T>
__device__ __forceinline__ T pending_inc(long long t, double scale, bool exact32) {
  if (sizeof(T) == 4 && exact32) return (T)(__ll2float_rn(t) * (float)scale);
  return (T)((double)t * scale);
}
//
// tx, ty: the thread's place in the 34 x (TY + 2) block; live == false for
// threads of a larger block that hold no site: they run the same code with
// every memory access switched off, so that all threads of a warp meet the
// same barrier instructions.  Sync is the barrier of the threads that run the
// tile.  The two
// updates are written as explicit fused multiply-adds, so the result does not
// depend on the compiler's contraction setting.
struct CtaSync {
  __device__ void operator()() const { __syncthreads(); }
};

template <typename T>
__device__ __forceinline__ T fma_t(T a, T b, T c);
template <>
__device__ __forceinline__ float fma_t<float>(float a, float b, float c) { return __fmaf_rn(a, b, c); }
template <>
__device__ __forceinline__ double fma_t<double>(double a, double b, double c) { return __fma_rn(a, b, c); }

template <typename T, int TY, int PF, class Sync, int TX = 32>
__device__ __forceinline__ void site_tile(const Mesh& m, const T* __restrict__ Din,
                                          const T* __restrict__ Bin, const T* __restrict__ ie,
                                          T* __restrict__ Dout, T* __restrict__ Bout, T cB, T cD,
                                          int tile_x, int tile_y, int tile_z, int zchunk, int tx,
                                          int ty, bool live, Sync sync,
                                          const long long* __restrict__ Tp = nullptr,
                                          double tscale = 0.0, bool exact32 = false) {
  static_assert(PF >= 1 && PF <= 2, "prefetch depth");
  static_assert(TX == 16 || TX == 32, "tile width");
  constexpr int EX = TX + 2, EY = TY + 2;
  __shared__ T sE[3][3][EY][EX];
  __shared__ T sB[2][3][EY][EX];
  const int nx = m.n[0], ny = m.n[1], nz = m.n[2];
  const int64_t V = m.V;
  const int64_t P = (int64_t)nx * ny;
  const int x0 = tile_x * TX, y0 = tile_y * TY;
  const int z0 = tile_z * zchunk;
  const int z1 = min(z0 + zchunk, nz);
  int x = x0 - 1 + tx, y = y0 - 1 + ty;
  const bool inside = live && tx >= 1 && tx <= TX && ty >= 1 && ty <= TY && x < nx && y < ny;
  const bool bel = live && tx <= TX && ty <= TY;  // B' computed here (tile and low halo)
  x = (x < 0) ? x + nx : (x >= nx ? x - nx : x);
  y = (y < 0) ? y + ny : (y >= ny ? y - ny : y);
  if (x >= nx) x = nx - 1;  // tiles wider than the mesh (unused values)
  if (y >= ny) y = ny - 1;
  const int64_t off = (int64_t)y * nx + x;
  // planes z0-1 .. z1 are touched: one wrap at either end is enough
  auto wrapz = [&](int k) { return k >= nz ? k - nz : (k < 0 ? k + nz : k); };
  auto ld3 = [&](const T* a, int k, T (&r)[3]) {
    if (!live) return;
    const T* p = a + (int64_t)k * P + off;
    r[0] = p[0];
    r[1] = p[V];
    r[2] = p[2 * V];
  };
  auto ldD = [&](int k, T (&r)[3]) {
    ld3(Din, k, r);
    if (!live || !Tp) return;
    const long long* q = Tp + tw_index(0, (int64_t)k * P + off, V);
#pragma unroll
    for (int c = 0; c < 3; ++c) {
      const long long t = q[c * V];
      if (t != 0) r[c] = r[c] + pending_inc<T>(t, tscale, exact32);
    }
  };
  auto putE = [&](int slot, const T (&d)[3], const T (&i)[3]) {
    if (!live) return;
    sE[slot][0][ty][tx] = d[0] * i[0];
    sE[slot][1][ty][tx] = d[1] * i[1];
    sE[slot][2][ty][tx] = d[2] * i[2];
  };
  auto compute_B = [&](int k, int ec, int en, int slot, const T (&bb)[3], bool store) {
    if (!bel) return;
    const T Ex = sE[ec][0][ty][tx], Ey = sE[ec][1][ty][tx], Ez = sE[ec][2][ty][tx];
    const T Ey_x = sE[ec][1][ty][tx + 1], Ez_x = sE[ec][2][ty][tx + 1];
    const T Ex_y = sE[ec][0][ty + 1][tx], Ez_y = sE[ec][2][ty + 1][tx];
    const T Ex_z = sE[en][0][ty][tx], Ey_z = sE[en][1][ty][tx];
    const T bxv = fma_t<T>(-cB, ((Ey + Ez_y) - Ey_z) - Ez, bb[0]);
    const T byv = fma_t<T>(-cB, ((Ez + Ex_z) - Ez_x) - Ex, bb[1]);
    const T bzv = fma_t<T>(-cB, ((Ex + Ey_x) - Ex_y) - Ey, bb[2]);
    sB[slot][0][ty][tx] = bxv;
    sB[slot][1][ty][tx] = byv;
    sB[slot][2][ty][tx] = bzv;
    if (store && inside) {
      T* p = Bout + (int64_t)k * P + off;
      p[0] = bxv;
      p[V] = byv;
      p[2 * V] = bzv;
    }
  };

  // register queues at the top of iteration k: dq[j] = D(k+j), j = 0..PF+1;
  // iq[j] = 1/eps(k+2+j), j = 0..PF-1; bq[j] = B(k+j), j = 0..PF
  T dq[PF + 2][3], iq[PF][3], bq[PF + 1][3];
#pragma unroll
  for (int j = 0; j < PF + 2; ++j) dq[j][0] = dq[j][1] = dq[j][2] = T(0);
#pragma unroll
  for (int j = 0; j < PF; ++j) iq[j][0] = iq[j][1] = iq[j][2] = T(0);
#pragma unroll
  for (int j = 0; j < PF + 1; ++j) bq[j][0] = bq[j][1] = bq[j][2] = T(0);
  {
    T dm[3] = {}, im[3] = {}, bm[3] = {}, i0[3] = {}, i1[3] = {};
    const int zm = wrapz(z0 - 1), zp = wrapz(z0 + 1);
    ldD(zm, dm);
    ld3(ie, zm, im);
    ld3(Bin, zm, bm);
    ldD(z0, dq[0]);
    ld3(ie, z0, i0);
    ld3(Bin, z0, bq[0]);
    ldD(zp, dq[1]);
    ld3(ie, zp, i1);
#pragma unroll
    for (int j = 0; j + 1 < PF; ++j)  // planes z0+2 .. z0+PF
      if (z0 + 2 + j <= z1) {
        ldD(wrapz(z0 + 2 + j), dq[2 + j]);
        ld3(ie, wrapz(z0 + 2 + j), iq[j]);
      }
#pragma unroll
    for (int j = 1; j < PF; ++j)  // planes z0+1 .. z0+PF-1
      if (z0 + j < z1) ld3(Bin, wrapz(z0 + j), bq[j]);
    putE(0, dm, im);
    putE(1, dq[0], i0);
    putE(2, dq[1], i1);
    sync();
    compute_B(zm, 0, 1, 0, bm, false);
  }
  int ec = 1, en = 2, ef = 0, bp = 0, bcs = 1;
  for (int k = z0; k < z1; ++k) {
    // issue plane k+PF+1 of D and 1/eps, plane k+PF of B
    if (k + PF + 1 <= z1) {
      ldD(wrapz(k + PF + 1), dq[PF + 1]);
      ld3(ie, wrapz(k + PF + 1), iq[PF - 1]);
    }
    if (k + PF < z1) ld3(Bin, wrapz(k + PF), bq[PF]);
    sync();  // E(k+1) stored, sB[bcs] free
    compute_B(k, ec, en, bcs, bq[0], true);
    sync();
    if (inside) {
      const T Bx = sB[bcs][0][ty][tx], By = sB[bcs][1][ty][tx], Bz = sB[bcs][2][ty][tx];
      T* p = Dout + (int64_t)k * P + off;
      p[0] = fma_t<T>(cD, ((Bz - sB[bcs][2][ty - 1][tx]) - By) + sB[bp][1][ty][tx], dq[0][0]);
      p[V] = fma_t<T>(cD, ((Bx - sB[bp][0][ty][tx]) - Bz) + sB[bcs][2][ty][tx - 1], dq[0][1]);
      p[2 * V] = fma_t<T>(cD, ((By - sB[bcs][1][ty][tx - 1]) - Bx) + sB[bcs][0][ty - 1][tx],
                          dq[0][2]);
    }
    if (k + 1 < z1) putE(ef, dq[2], iq[0]);  // E(k+2), read from the next iteration on
#pragma unroll
    for (int j = 0; j < PF + 1; ++j)
#pragma unroll
      for (int c = 0; c < 3; ++c) dq[j][c] = dq[j + 1][c];
#pragma unroll
    for (int j = 0; j + 1 < PF; ++j)
#pragma unroll
      for (int c = 0; c < 3; ++c) iq[j][c] = iq[j + 1][c];
#pragma unroll
    for (int j = 0; j < PF; ++j)
#pragma unroll
      for (int c = 0; c < 3; ++c) bq[j][c] = bq[j + 1][c];
    const int t = ec;
    ec = en;
    en = ef;
    ef = t;
    bp ^= 1;
    bcs ^= 1;
  }
}

}  // namespace memd
