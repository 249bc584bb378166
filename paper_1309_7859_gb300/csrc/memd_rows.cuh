// memd_rows.cuh -- the row kernel's segment update (Eq. 20 a-b over whole
// lattice rows of 16-byte vectors), shared by the batched row kernel
// (memd_rows.cu) and the single-launch batch step (memd_particles.cu).
//
// A tile spans the full x extent of the mesh, so x needs no halo (the row is
// periodic in shared memory) and every global access is a 16-byte vector.  A
// tile is Rt rows plus one halo row below (its B' feeds the first row's D')
// and one above (its E feeds the last row's B'); it streams through a range
// of planes with the plane ahead in registers, one shared plane of E and one
// of B', and two barriers a plane.  Arithmetic per site is that of the other
// field kernels, term for term, so the result is bit identical to them.
#pragma once

#include "memd_internal.cuh"

namespace memd {
namespace rows {

template <typename T>
struct V16;
template <>
struct V16<float> {
  using V = float4;
  static constexpr int W = 4;
};
template <>
struct V16<double> {
  using V = double2;
  static constexpr int W = 2;
};

template <typename T>
__device__ __forceinline__ T fmat(T a, T b, T c);
template <>
__device__ __forceinline__ float fmat<float>(float a, float b, float c) { return __fmaf_rn(a, b, c); }
template <>
__device__ __forceinline__ double fmat<double>(double a, double b, double c) { return __fma_rn(a, b, c); }

// a 16-byte vector as W values and back
template <typename T>
struct Pack {
  T v[V16<T>::W];
};
__device__ __forceinline__ Pack<float> unpack(const float4& a) { return Pack<float>{{a.x, a.y, a.z, a.w}}; }
__device__ __forceinline__ Pack<double> unpack(const double2& a) { return Pack<double>{{a.x, a.y}}; }
__device__ __forceinline__ float4 repack(const Pack<float>& p) {
  return make_float4(p.v[0], p.v[1], p.v[2], p.v[3]);
}
__device__ __forceinline__ double2 repack(const Pack<double>& p) { return make_double2(p.v[0], p.v[1]); }

// per-thread asynchronous 16-byte copy global -> shared (L2 only), and its
// group bookkeeping.  The stencil reads and writes each field word once a
// step: its copies, loads and stores carry the evict_first policy, so that
// they do not push the particle kernels' transfer words out of L2.
__device__ __forceinline__ void cp_async16(void* smem, const void* gmem) {
  const unsigned sa = (unsigned)__cvta_generic_to_shared(smem);
  asm volatile("cp.async.cg.shared.global.L2::cache_hint [%0], [%1], 16, %2;" ::"r"(sa),
               "l"(gmem), "l"(l2_policy_first())
               : "memory");
}
__device__ __forceinline__ float4 ldcg_first(const float4* a) {
  float4 v;
  asm volatile("ld.global.cg.L2::cache_hint.v4.f32 {%0,%1,%2,%3}, [%4], %5;"
               : "=f"(v.x), "=f"(v.y), "=f"(v.z), "=f"(v.w)
               : "l"(a), "l"(l2_policy_first()));
  return v;
}
__device__ __forceinline__ double2 ldcg_first(const double2* a) {
  double2 v;
  asm volatile("ld.global.cg.L2::cache_hint.v2.f64 {%0,%1}, [%2], %3;"
               : "=d"(v.x), "=d"(v.y)
               : "l"(a), "l"(l2_policy_first()));
  return v;
}
__device__ __forceinline__ void st_first(float4* a, const float4& v) {
  asm volatile("st.global.L2::cache_hint.v4.f32 [%0], {%1,%2,%3,%4}, %5;" ::"l"(a), "f"(v.x),
               "f"(v.y), "f"(v.z), "f"(v.w), "l"(l2_policy_first())
               : "memory");
}
__device__ __forceinline__ void st_first(double2* a, const double2& v) {
  asm volatile("st.global.L2::cache_hint.v2.f64 [%0], {%1,%2}, %3;" ::"l"(a), "d"(v.x), "d"(v.y),
               "l"(l2_policy_first())
               : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
template <int N>
__device__ __forceinline__ void cp_async_wait() {
  asm volatile("cp.async.wait_group %0;" ::"n"(N) : "memory");
}

// One segment: replica mesh m, rows y0 .. y0 + Rt - 1 of planes za .. zb - 1.
// Thread t holds row r = t / TQ of the tile (r = 0: the halo row y0 - 1,
// r = Rt + 1: the halo row y0 + Rt) and sites x = W (t % TQ) .. + W - 1.
// Threads beyond the tile's rows only take part in the barriers.
template <typename T, int NT>
__device__ __forceinline__ void rows_segment(const Mesh& m, const T* __restrict__ Din,
                                             const T* __restrict__ Bin, const T* __restrict__ ie,
                                             T* __restrict__ Dout, T* __restrict__ Bout, T cB,
                                             T cD, int y0, int Rt, int za, int zb, T* sE,
                                             T* sB, unsigned char* stg) {
  using VT = typename V16<T>::V;
  constexpr int W = V16<T>::W;
  const int nx = m.n[0], ny = m.n[1], nz = m.n[2];
  const int64_t V = m.V;
  const int64_t P = (int64_t)nx * ny;
  const int TQ = nx / W;
  const int rows = Rt + 2;
  const int t = threadIdx.x;
  const int r = t / TQ;
  const int xq = t - r * TQ;
  const bool act = r < rows;
  const bool doB = act && r <= Rt;              // B' here (tile and low halo)
  const bool doD = act && r >= 1 && r <= Rt;   // D' here (tile rows)
  int y = y0 - 1 + r;
  y = y < 0 ? y + ny : (y >= ny ? y - ny : y);
  const int x = xq * W;
  const int64_t off = (int64_t)y * nx + x;
  // shared planes: component c, tile row rr, site xx at (c rows + rr) nx + xx
  const int plane = rows * nx;
  const int s0 = r * nx + x;                                  // own first site
  const int sxp = r * nx + (xq + 1 == TQ ? 0 : x + W);        // site x + W (wrapped)
  const int sxm = r * nx + (xq == 0 ? nx - 1 : x - 1);        // site x - 1 (wrapped)
  const int syp = (r + 1) * nx + x;                           // row above
  const int sym = (r - 1) * nx + x;                           // row below
  auto wrapz = [&](int k) { return k >= nz ? k - nz : (k < 0 ? k + nz : k); };
  auto ld = [&](const T* a, int k, int c) {
    return unpack(__ldg(reinterpret_cast<const VT*>(a + (int64_t)c * V + (int64_t)k * P + off)));
  };
  auto ldcg = [&](const T* a, int k, int c) {
    return unpack(ldcg_first(reinterpret_cast<const VT*>(a + (int64_t)c * V + (int64_t)k * P + off)));
  };
  auto st = [&](T* a, int k, int c, const Pack<T>& v) {
    st_first(reinterpret_cast<VT*>(a + (int64_t)c * V + (int64_t)k * P + off), repack(v));
  };
  auto sput = [&](T* s, int c, const Pack<T>& v) {
    *reinterpret_cast<VT*>(s + c * plane + s0) = repack(v);
  };

  // B' of plane k at the thread's sites: E(k) in sE (own, x + 1, y + 1),
  // E(k + 1) own (En), B(k) own (Bo)
  auto curlE = [&](const Pack<T> (&En)[3], const Pack<T> (&Bo)[3], Pack<T> (&Bn)[3]) {
    const Pack<T> Ex = unpack(*reinterpret_cast<const VT*>(sE + 0 * plane + s0));
    const Pack<T> Ey = unpack(*reinterpret_cast<const VT*>(sE + 1 * plane + s0));
    const Pack<T> Ez = unpack(*reinterpret_cast<const VT*>(sE + 2 * plane + s0));
    const Pack<T> Exy = unpack(*reinterpret_cast<const VT*>(sE + 0 * plane + syp));
    const Pack<T> Ezy = unpack(*reinterpret_cast<const VT*>(sE + 2 * plane + syp));
    const T Eyx = sE[1 * plane + sxp], Ezx = sE[2 * plane + sxp];
#pragma unroll
    for (int j = 0; j < W; ++j) {
      const T ey_x = j + 1 < W ? Ey.v[j + 1] : Eyx;
      const T ez_x = j + 1 < W ? Ez.v[j + 1] : Ezx;
      Bn[0].v[j] = fmat<T>(-cB, ((Ey.v[j] + Ezy.v[j]) - En[1].v[j]) - Ez.v[j], Bo[0].v[j]);
      Bn[1].v[j] = fmat<T>(-cB, ((Ez.v[j] + En[0].v[j]) - ez_x) - Ex.v[j], Bo[1].v[j]);
      Bn[2].v[j] = fmat<T>(-cB, ((Ex.v[j] + ey_x) - Exy.v[j]) - Ey.v[j], Bo[2].v[j]);
    }
  };
  // D' of plane k: B'(k) in sB (own, x - 1, y - 1), B'(k - 1) own (Bm)
  auto curlB = [&](const Pack<T> (&Bm)[3], const Pack<T> (&Dk)[3], Pack<T> (&Dn)[3]) {
    const Pack<T> Bx = unpack(*reinterpret_cast<const VT*>(sB + 0 * plane + s0));
    const Pack<T> By = unpack(*reinterpret_cast<const VT*>(sB + 1 * plane + s0));
    const Pack<T> Bz = unpack(*reinterpret_cast<const VT*>(sB + 2 * plane + s0));
    const Pack<T> Bxy = unpack(*reinterpret_cast<const VT*>(sB + 0 * plane + sym));
    const Pack<T> Bzy = unpack(*reinterpret_cast<const VT*>(sB + 2 * plane + sym));
    const T Byx = sB[1 * plane + sxm], Bzx = sB[2 * plane + sxm];
#pragma unroll
    for (int j = 0; j < W; ++j) {
      const T by_x = j > 0 ? By.v[j - 1] : Byx;
      const T bz_x = j > 0 ? Bz.v[j - 1] : Bzx;
      Dn[0].v[j] = fmat<T>(cD, ((Bz.v[j] - Bzy.v[j]) - By.v[j]) + Bm[1].v[j], Dk[0].v[j]);
      Dn[1].v[j] = fmat<T>(cD, ((Bx.v[j] - Bm[0].v[j]) - Bz.v[j]) + bz_x, Dk[1].v[j]);
      Dn[2].v[j] = fmat<T>(cD, ((By.v[j] - by_x) - Bx.v[j]) + Bxy.v[j], Dk[2].v[j]);
    }
  };
  auto mulE = [&](const Pack<T> (&d)[3], const Pack<T> (&i)[3], Pack<T> (&e)[3]) {
#pragma unroll
    for (int c = 0; c < 3; ++c)
#pragma unroll
      for (int j = 0; j < W; ++j) e[c].v[j] = d[c].v[j] * i[c].v[j];
  };

  // D and 1/eps of three planes are staged in shared memory by per-thread
  // asynchronous 16-byte copies (each thread copies and later reads only
  // its own vectors), so two planes stay in flight without holding
  // registers; B of the next plane is loaded into registers.  The slot of
  // plane p is (p - za + 1) mod 3.
  auto slot_ptr = [&](int slot, int f, int c) {
    return stg + ((size_t)((slot * 6 + f * 3 + c) * NT + t)) * 16;
  };
  auto issue = [&](int p, int slot) {
    if (act) {
      const int kp = wrapz(p);
#pragma unroll
      for (int c = 0; c < 3; ++c) {
        cp_async16(slot_ptr(slot, 0, c), Din + (int64_t)c * V + (int64_t)kp * P + off);
        cp_async16(slot_ptr(slot, 1, c), ie + (int64_t)c * V + (int64_t)kp * P + off);
      }
    }
    cp_async_commit();
  };
  auto rd = [&](int slot, int f, int c) {
    return unpack(*reinterpret_cast<const VT*>(slot_ptr(slot, f, c)));
  };

  Pack<T> Bq[3], Bm[3], En[3];
  // prologue: E(za - 1) shared, E(za) own, B'(za - 1) own
  {
    issue(za - 1, 0);
    issue(za, 1);
    issue(za + 1, 2);  // za + 1 <= zb: D(zb) is needed for E(zb)
    Pack<T> bm[3];
    if (act) {
      const int zm = wrapz(za - 1);
#pragma unroll
      for (int c = 0; c < 3; ++c) {
        bm[c] = ldcg(Bin, zm, c);
        Bq[c] = ldcg(Bin, za, c);
      }
    }
    cp_async_wait<1>();  // planes za - 1 and za
    if (act) {
      Pack<T> d[3], i[3], Em[3];
#pragma unroll
      for (int c = 0; c < 3; ++c) {
        d[c] = rd(0, 0, c);
        i[c] = rd(0, 1, c);
      }
      mulE(d, i, Em);
#pragma unroll
      for (int c = 0; c < 3; ++c) {
        sput(sE, c, Em[c]);
        d[c] = rd(1, 0, c);
        i[c] = rd(1, 1, c);
      }
      mulE(d, i, En);
    }
    __syncthreads();
    if (doB) curlE(En, bm, Bm);
    __syncthreads();
    if (act)
#pragma unroll
      for (int c = 0; c < 3; ++c) sput(sE, c, En[c]);
    // plane za - 1's slot takes plane za + 2
    if (za + 2 <= zb)
      issue(za + 2, 0);
    else
      cp_async_commit();
    __syncthreads();
  }
  for (int k = za; k < zb; ++k) {
    // E(k) is in sE; D(k) staged; D(k + 1), 1/eps(k + 1) staged or
    // arriving (plane k + 2 may still be in flight); B(k) in Bq
    const int sk = (k - za + 1) % 3, sk1 = (k - za + 2) % 3;
    cp_async_wait<1>();
    Pack<T> Bo[3];
#pragma unroll
    for (int c = 0; c < 3; ++c) Bo[c] = Bq[c];
    if (act) {
      Pack<T> d[3], i[3];
#pragma unroll
      for (int c = 0; c < 3; ++c) {
        d[c] = rd(sk1, 0, c);
        i[c] = rd(sk1, 1, c);
      }
      mulE(d, i, En);  // E(k + 1) own
    }
    Pack<T> Bn[3];
    if (doB) {
      curlE(En, Bo, Bn);
#pragma unroll
      for (int c = 0; c < 3; ++c) sput(sB, c, Bn[c]);
      if (doD)
#pragma unroll
        for (int c = 0; c < 3; ++c) st(Bout, k, c, Bn[c]);
    }
    if (act && k + 1 < zb) {
      const int z1 = wrapz(k + 1);
#pragma unroll
      for (int c = 0; c < 3; ++c) Bq[c] = ldcg(Bin, z1, c);
    }
    __syncthreads();  // B'(k) shared; every read of E(k) done
    if (act)
#pragma unroll
      for (int c = 0; c < 3; ++c) sput(sE, c, En[c]);
    if (doD) {
      Pack<T> Dk[3], Dn[3];
#pragma unroll
      for (int c = 0; c < 3; ++c) Dk[c] = rd(sk, 0, c);
      curlB(Bm, Dk, Dn);
#pragma unroll
      for (int c = 0; c < 3; ++c) st(Dout, k, c, Dn[c]);
    }
#pragma unroll
    for (int c = 0; c < 3; ++c) Bm[c] = Bn[c];
    __syncthreads();  // E(k + 1) shared; every read of B'(k) and of plane k done
    // plane k's slot takes plane k + 3
    if (k + 3 <= zb)
      issue(k + 3, sk);
    else
      cp_async_commit();
  }
  cp_async_wait<0>();
}

}  // namespace rows
}  // namespace memd
