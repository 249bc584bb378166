// memd_site.cuh -- the one-thread-per-site fused field update (B' from the
// circulation of E = D / eps, then D' from the curl of B', Eq. 20 a-b),
// shared by the field kernels and the single-launch step kernel.
#pragma once
#include <utility>

#include "memd_internal.cuh"

namespace memd {

// Fused field update, one thread per site of the tile and of its halo ring.
// A CTA of 34 x (TY + 2) threads covers the 32 x TY tile plus one site on
// every side.  Each thread loads D, 1/eps and B of its own site only (nine
// values a plane, one base pointer), writes its E = D / eps into the shared
// ring of planes k, k+1, k+2, computes B' at its site (tile and low halo),
// and, inside the tile, D' from its own D kept in registers.  Loads run PF
// planes ahead of the plane being computed, so that about 9 PF values per
// thread are in flight while a plane is computed.  Same arithmetic per site
// as k_fused_curl.
//
// The z loop is unrolled over the common period of all rings (the three E
// planes, the two B' planes and the register queues of D, 1/eps and B), so
// that every ring slot is a compile-time index: no register moves between
// planes and no computed shared-memory addresses.  Offsets are 32-bit (a
// context holds fewer than 2^31 links).
//
// tx, ty: the thread's place in the 34 x (TY + 2) block; live == false for
// threads of a larger block that hold no site: they run the same code with
// every memory access switched off, so that all threads of a warp meet the
// same barrier instructions.  Sync is the barrier of the threads that run the
// tile.  The two updates are written as explicit fused multiply-adds, so the
// result does not depend on the compiler's contraction setting.
struct CtaSync {
  __device__ void operator()() const { __syncthreads(); }
};

template <typename T>
__device__ __forceinline__ T fma_t(T a, T b, T c);
template <>
__device__ __forceinline__ float fma_t<float>(float a, float b, float c) { return __fmaf_rn(a, b, c); }
template <>
__device__ __forceinline__ double fma_t<double>(double a, double b, double c) { return __fma_rn(a, b, c); }

constexpr int site_gcd(int a, int b) { return b == 0 ? a : site_gcd(b, a % b); }
constexpr int site_lcm(int a, int b) { return a / site_gcd(a, b) * b; }

template <typename T, int TY, int PF, class Sync>
struct SiteTile {
  static_assert(PF >= 1 && PF <= 2, "prefetch depth");
  static constexpr int TX = 32, EX = TX + 2, EY = TY + 2;
  static constexpr int QD = PF + 2;  // D(k) .. D(k+PF+1)
  static constexpr int QI = PF;      // 1/eps(k+2) .. 1/eps(k+PF+1)
  static constexpr int QB = PF + 1;  // B(k) .. B(k+PF)
  // period of the unrolled loop: every ring returns to its first slot
  static constexpr int U = site_lcm(site_lcm(site_lcm(QD, QI), site_lcm(QB, 3)), 2);

  T (*sE)[3][EY][EX];  // E ring: 3 planes
  T (*sB)[3][EY][EX];  // B' ring: 2 planes
  const T* __restrict__ Din;
  const T* __restrict__ Bin;
  const T* __restrict__ ie;
  T* __restrict__ Dout;
  T* __restrict__ Bout;
  T cB, cD;
  int nz, z0, z1, P, V, off, tx, ty;
  bool live, inside, bel;
  Sync sync;
  T dq[QD][3], iq[QI][3], bq[QB][3];

  __device__ __forceinline__ int wrapz(int k) const {
    return k >= nz ? k - nz : (k < 0 ? k + nz : k);  // planes z0-1 .. z1 only
  }
  __device__ __forceinline__ void ld3(const T* a, int k, T (&r)[3]) const {
    if (!live) return;
    const T* p = a + (k * P + off);
    r[0] = p[0];
    r[1] = p[V];
    r[2] = p[2 * V];
  }
  __device__ __forceinline__ void putE(int slot, const T (&d)[3], const T (&i)[3]) {
    if (!live) return;
    sE[slot][0][ty][tx] = d[0] * i[0];
    sE[slot][1][ty][tx] = d[1] * i[1];
    sE[slot][2][ty][tx] = d[2] * i[2];
  }
  // B' of plane k from E in slots ec (k) and en (k+1) and B(k) in registers
  __device__ __forceinline__ void compute_B(int k, int ec, int en, int slot, const T (&bb)[3],
                                            bool store) {
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
      T* p = Bout + (k * P + off);
      p[0] = bxv;
      p[V] = byv;
      p[2 * V] = bzv;
    }
  }

  // iteration k = z0 + i with I = i mod U
  template <int I>
  __device__ __forceinline__ void plane(int k) {
    // issue plane k+PF+1 of D and 1/eps and plane k+PF of B
    if (k + PF + 1 <= z1) {
      ld3(Din, wrapz(k + PF + 1), dq[(I + PF + 1) % QD]);
      ld3(ie, wrapz(k + PF + 1), iq[(I + PF - 1) % QI]);
    }
    if (k + PF < z1) ld3(Bin, wrapz(k + PF), bq[(I + PF) % QB]);
    constexpr int ec = (I + 1) % 3, en = (I + 2) % 3, ef = I % 3;
    constexpr int bcs = (I + 1) % 2, bp = I % 2;
    sync();  // E(k+1) stored, sB[bcs] free
    compute_B(k, ec, en, bcs, bq[I % QB], true);
    sync();
    if (inside) {
      const T(&d0)[3] = dq[I % QD];
      const T Bx = sB[bcs][0][ty][tx], By = sB[bcs][1][ty][tx], Bz = sB[bcs][2][ty][tx];
      T* p = Dout + (k * P + off);
      p[0] = fma_t<T>(cD, ((Bz - sB[bcs][2][ty - 1][tx]) - By) + sB[bp][1][ty][tx], d0[0]);
      p[V] = fma_t<T>(cD, ((Bx - sB[bp][0][ty][tx]) - Bz) + sB[bcs][2][ty][tx - 1], d0[1]);
      p[2 * V] = fma_t<T>(cD, ((By - sB[bcs][1][ty][tx - 1]) - Bx) + sB[bcs][0][ty - 1][tx], d0[2]);
    }
    // E(k+2) into the slot of E(k-1), read from the next iteration on
    if (k + 1 < z1) putE(ef, dq[(I + 2) % QD], iq[I % QI]);
  }
  template <int... Is>
  __device__ __forceinline__ void period(int k, std::integer_sequence<int, Is...>) {
    (plane<Is>(k + Is), ...);
  }
  template <int... Is>
  __device__ __forceinline__ void tail(int k, std::integer_sequence<int, Is...>) {
    ((k + Is < z1 ? plane<Is>(k + Is) : void()), ...);
  }

  __device__ __forceinline__ void run() {
#pragma unroll
    for (int j = 0; j < QD; ++j) dq[j][0] = dq[j][1] = dq[j][2] = T(0);
#pragma unroll
    for (int j = 0; j < QI; ++j) iq[j][0] = iq[j][1] = iq[j][2] = T(0);
#pragma unroll
    for (int j = 0; j < QB; ++j) bq[j][0] = bq[j][1] = bq[j][2] = T(0);
    {
      // queues as iteration 0 expects them, E(z0-1), E(z0), E(z0+1) in
      // slots 0, 1, 2 and B'(z0-1) in slot 0
      T dm[3] = {}, im[3] = {}, bm[3] = {}, i0[3] = {}, i1[3] = {};
      const int zm = wrapz(z0 - 1), zp = wrapz(z0 + 1);
      ld3(Din, zm, dm);
      ld3(ie, zm, im);
      ld3(Bin, zm, bm);
      ld3(Din, z0, dq[0]);
      ld3(ie, z0, i0);
      ld3(Bin, z0, bq[0]);
      ld3(Din, zp, dq[1 % QD]);
      ld3(ie, zp, i1);
#pragma unroll
      for (int j = 0; j + 1 < PF; ++j)  // planes z0+2 .. z0+PF
        if (z0 + 2 + j <= z1) {
          ld3(Din, wrapz(z0 + 2 + j), dq[(2 + j) % QD]);
          ld3(ie, wrapz(z0 + 2 + j), iq[j % QI]);
        }
#pragma unroll
      for (int j = 1; j < PF; ++j)  // planes z0+1 .. z0+PF-1
        if (z0 + j < z1) ld3(Bin, wrapz(z0 + j), bq[j % QB]);
      putE(0, dm, im);
      putE(1, dq[0], i0);
      putE(2, dq[1 % QD], i1);
      sync();
      compute_B(zm, 0, 1, 0, bm, false);
    }
    int k = z0;
    for (; k + U <= z1; k += U) period(k, std::make_integer_sequence<int, U>{});
    if (k < z1) tail(k, std::make_integer_sequence<int, U - 1>{});
  }
};

template <typename T, int TY, int PF, class Sync>
__device__ __forceinline__ void site_tile(const Mesh& m, const T* __restrict__ Din,
                                          const T* __restrict__ Bin, const T* __restrict__ ie,
                                          T* __restrict__ Dout, T* __restrict__ Bout, T cB, T cD,
                                          int tile_x, int tile_y, int tile_z, int zchunk, int tx,
                                          int ty, bool live, Sync sync) {
  using Tile = SiteTile<T, TY, PF, Sync>;
  __shared__ T sE[3][3][Tile::EY][Tile::EX];
  __shared__ T sB[2][3][Tile::EY][Tile::EX];
  const int nx = m.n[0], ny = m.n[1];
  Tile t;
  t.sE = sE;
  t.sB = sB;
  t.Din = Din;
  t.Bin = Bin;
  t.ie = ie;
  t.Dout = Dout;
  t.Bout = Bout;
  t.cB = cB;
  t.cD = cD;
  t.nz = m.n[2];
  t.z0 = tile_z * zchunk;
  t.z1 = min(t.z0 + zchunk, t.nz);
  t.P = nx * ny;
  t.V = (int)m.V;
  t.tx = tx;
  t.ty = ty;
  t.live = live;
  t.sync = sync;
  int x = tile_x * Tile::TX - 1 + tx, y = tile_y * TY - 1 + ty;
  t.inside = live && tx >= 1 && tx <= Tile::TX && ty >= 1 && ty <= TY && x < nx && y < ny;
  t.bel = live && tx <= Tile::TX && ty <= TY;  // B' computed here (tile and low halo)
  x = (x < 0) ? x + nx : (x >= nx ? x - nx : x);
  y = (y < 0) ? y + ny : (y >= ny ? y - ny : y);
  if (x >= nx) x = nx - 1;  // tiles wider than the mesh (unused values)
  if (y >= ny) y = ny - 1;
  t.off = y * nx + x;
  t.run();
}

}  // namespace memd
