// memd_rows.cu -- fused field update (Eq. 20 a-b: B' from the circulation
// of E = D / eps, then D' from the curl of B') over whole lattice rows, for
// the batched replicas.
//
// Small and medium meshes make the one-thread-per-site tile pay for its halo
// columns and for its instruction count: the stencil is issue bound there.
// This kernel gives each thread W consecutive sites of a row (one 16-byte
// vector: 4 FP32 or 2 FP64 values a component), and a tile spans the full x
// extent of the mesh, so x needs no halo (the row is periodic in shared
// memory) and every global access is a 16-byte vector.  A tile is Rt rows
// plus one halo row below (its B' feeds the first row's D') and one above
// (its E feeds the last row's B'); it streams through a range of planes
// with the plane ahead in registers, one shared plane of E and one of B',
// and two barriers a plane.
//
// Work balance: the host cuts all tile-planes of all replicas, weighted by
// their cost, into one contiguous range per CTA of a
// persistent grid (occupancy x SMs); a range is a list of segments (replica,
// tile, planes).  Every CTA then carries the same load, whatever the mix of
// mesh sizes, and there is no tail wave.
//
// Arithmetic per site is that of the other field kernels, term for term, so
// the result is bit identical to them.
#include <algorithm>
#include <vector>

#include "memd_ctx.cuh"
#include "memd_internal.cuh"

namespace memd {

namespace {

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
// group bookkeeping
__device__ __forceinline__ void cp_async16(void* smem, const void* gmem) {
  const unsigned sa = (unsigned)__cvta_generic_to_shared(smem);
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(sa), "l"(gmem) : "memory");
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
    return unpack(__ldcg(reinterpret_cast<const VT*>(a + (int64_t)c * V + (int64_t)k * P + off)));
  };
  auto st = [&](T* a, int k, int c, const Pack<T>& v) {
    *reinterpret_cast<VT*>(a + (int64_t)c * V + (int64_t)k * P + off) = repack(v);
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

struct RowsArgs {
  const RepDesc* desc;
  const RowSeg* segs;
  const int* seg_first;
  int par;
};

// two CTAs of 256 threads or one of 512 an SM (shared memory)
template <typename T, int NT>
__global__ void __launch_bounds__(NT, NT >= 512 ? 1 : 2) k_rows_batch(const __grid_constant__ RowsArgs a) {
  extern __shared__ __align__(16) unsigned char rows_smem[];
  const int s_end = a.seg_first[blockIdx.x + 1];
  for (int s = a.seg_first[blockIdx.x]; s < s_end; ++s) {
    const RowSeg g = a.segs[s];
    const RepDesc& r = a.desc[g.rep];
    // the staged planes (3 slots x D, 1/eps x 3 components x NT vectors),
    // then the shared E and B' planes sized for this tile: 3 rows nx each
    const int plane3 = 3 * (g.rows + 2) * r.m.n[0];
    unsigned char* stg = rows_smem;
    T* sE = reinterpret_cast<T*>(rows_smem + (size_t)3 * 6 * NT * 16);
    T* sB = sE + plane3;
    rows_segment<T, NT>(r.m, (const T*)r.D[a.par], (const T*)r.B[a.par], (const T*)r.ie,
                        (T*)r.D[a.par ^ 1], (T*)r.B[a.par ^ 1], (T)r.sp.coefB, (T)r.sp.coefD,
                        g.y0, g.rows, g.za, g.zb, sE, sB, stg);
  }
}

// the kernel's dynamic shared memory exceeds the 48 KB default: raise its
// limit (once per process and instantiation) before any launch or
// occupancy query
template <typename T, int NT>
cudaError_t rows_attr() {
  static cudaError_t done = cudaFuncSetAttribute(
      k_rows_batch<T, NT>, cudaFuncAttributeMaxDynamicSharedMemorySize,
      (int)rows_smem_bytes(NT, sizeof(T)));
  return done;
}

template <typename T, int NT>
cudaError_t rows_launch(const RowsArgs& a, int nctas, cudaStream_t st) {
  const cudaError_t e = rows_attr<T, NT>();
  if (e != cudaSuccess) return e;
  k_rows_batch<T, NT><<<nctas, NT, rows_smem_bytes(NT, sizeof(T)), st>>>(a);
  return cudaGetLastError();
}

template <typename T, int NT>
int rows_occ() {
  int n = 0;
  if (rows_attr<T, NT>() != cudaSuccess ||
      cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, k_rows_batch<T, NT>, NT,
                                                    rows_smem_bytes(NT, sizeof(T))) !=
          cudaSuccess) {
    cudaGetLastError();
    return 0;
  }
  return n;
}

}  // namespace

size_t rows_smem_bytes(int nt, size_t esz) {
  // three staged planes of D and 1/eps (6 vectors of 16 bytes a thread),
  // then the E and B' planes of 3 components; a tile holds at most nt
  // threads of 16 bytes of sites each, whatever the element size
  (void)esz;
  return (3 * 6 + 2 * 3) * (size_t)nt * 16;
}

int rows_sites_per_thread(int prec) { return prec == 1 ? 4 : 2; }

int rows_occupancy(int prec, int nt) {
  if (prec == 1) return nt == 256 ? rows_occ<float, 256>() : rows_occ<float, 512>();
  return nt == 256 ? rows_occ<double, 256>() : rows_occ<double, 512>();
}

cudaError_t launch_rows_batch(int prec, const RepDesc* desc, const RowSeg* segs,
                              const int* seg_first, int nctas, int nt, int par, cudaStream_t st) {
  if (nctas <= 0) return cudaSuccess;
  const RowsArgs a{desc, segs, seg_first, par};
  if (prec == 1) return nt == 256 ? rows_launch<float, 256>(a, nctas, st) : rows_launch<float, 512>(a, nctas, st);
  return nt == 256 ? rows_launch<double, 256>(a, nctas, st) : rows_launch<double, 512>(a, nctas, st);
}

// cost model of the row plan (measured on 64 mixed replicas): a tile-plane
// costs no less than 256 threads' worth of vectors, the latency of one plane
// in flight that small tiles cannot cover; a segment's prologue costs two
// planes
constexpr long long kRowsFloor = 256;
constexpr long long kRowsPro = 2;
bool rows_plan(const std::vector<memd_ctx*>& m, int prec, int nt, int nctas,
               std::vector<RowSeg>& segs, std::vector<int>& first) {
  const int W = rows_sites_per_thread(prec);
  struct Tile {
    int rep, y0, rows, nz;
    long long w;
  };
  std::vector<Tile> tiles;
  for (size_t r = 0; r < m.size(); ++r) {
    const memd_ctx* c = m[r];
    const int nx = c->mesh.n[0], ny = c->mesh.n[1], nz = c->mesh.n[2];
    if (nx % W != 0) return false;
    for (int t = 0; t < 2; ++t)
      if (((uintptr_t)c->Dbuf[t] | (uintptr_t)c->Bbuf[t]) % 16 != 0) return false;
    if ((uintptr_t)c->ie % 16 != 0) return false;
    const int TQ = nx / W;
    const int maxrows = nt / TQ;
    if (maxrows < 3) return false;
    const int ntl = (ny + maxrows - 3) / (maxrows - 2);
    const int Rt = (ny + ntl - 1) / ntl;
    for (int y0 = 0; y0 < ny; y0 += Rt) {
      const int rows = std::min(Rt, ny - y0);
      // a tile-plane costs its bytes (threads x 16-byte vectors) once the
      // memory pipe is full, but no less than kRowsFloor
      const long long w = std::max<long long>(TQ * (rows + 2), kRowsFloor);
      tiles.push_back(Tile{(int)r, y0, rows, nz, w});
    }
  }
  // Greedy cut in order with a capacity per CTA: a segment's first plane
  // also pays its prologue (the plane below and the wait for the first
  // planes), `pro` planes' worth.  The capacity is the least for which the
  // greedy cut needs no more than nctas CTAs (bisection).
  const long long pro = kRowsPro;
  auto cut = [&](long long cap, bool build) {
    int cta = 0;
    long long load = 0;
    bool open = false;  // the current CTA holds a segment
    if (build) {
      segs.clear();
      first.assign(nctas + 1, 0);
    }
    int last_rep = -1, last_y0 = -1, last_zb = -1;
    for (const Tile& t : tiles) {
      for (int k = 0; k < t.nz; ++k) {
        const bool cont = open && last_rep == t.rep && last_y0 == t.y0 && last_zb == k;
        long long cost = t.w + (cont ? 0 : pro * t.w);
        bool fresh = !cont;
        if (open && load + cost > cap) {  // close this CTA
          ++cta;
          if (build && cta <= nctas) first[cta] = (int)segs.size();
          load = 0;
          cost = t.w + pro * t.w;
          fresh = true;
        }
        if (build && cta < nctas) {
          if (fresh)
            segs.push_back(RowSeg{t.rep, t.y0, t.rows, k, k + 1});
          else
            segs.back().zb = k + 1;
        }
        open = true;
        load += cost;
        last_rep = t.rep;
        last_y0 = t.y0;
        last_zb = k + 1;
      }
    }
    if (build)
      while (cta < nctas) first[++cta] = (int)segs.size();
    return cta + 1;  // CTAs used
  };
  long long lo = 1, hi = 0;
  for (const Tile& t : tiles) hi += (long long)t.nz * t.w + pro * t.w * (long long)t.nz;
  while (lo < hi) {
    const long long mid = lo + (hi - lo) / 2;
    if (cut(mid, false) <= nctas)
      hi = mid;
    else
      lo = mid + 1;
  }
  cut(lo, true);
  return true;
}

}  // namespace memd
