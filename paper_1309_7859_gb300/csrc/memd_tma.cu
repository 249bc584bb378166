// memd_tma.cu -- the fused field update of one step (Eqs. 20 and 21 without
// the current) with TMA-staged planes, for meshes whose x rows are 16-byte
// multiples.
//
// Each CTA owns a 32 x TY column tile and marches up a chunk of z planes.
// One 4-D TMA box per array brings a plane tile of D, 1/eps and B (all three
// components, x from x0 - HP to x0 + 32 + HP, y from y0 - 1 to y0 + TY)
// into shared memory; NS such planes are kept in a ring guarded by
// mbarriers, so the copy engine fetches two planes ahead while the threads
// compute B' = B - cB circ(D ie) on the tile plus its low halo and then
// D' = D + cD (transpose circulation of B').  The copy engine generates all
// addresses; the threads only do the stencil arithmetic.  TMA does not wrap
// periodically, so CTAs on the mesh boundary patch their halo ring from the
// opposite side with plain loads.  Every mbarrier wait is bounded by a clock
// budget: on timeout the kernel raises kErrTimeout, drains its own copies
// (also bounded) and returns, never hanging the GPU.
#include <cudaTypedefs.h>

#include "memd_internal.cuh"

namespace memd {

namespace {

constexpr long long kWaitBudget = 200000000ll;  // SM clocks (~0.1 s) per wait

__device__ inline unsigned smem_u32(const void* p) {
  return (unsigned)__cvta_generic_to_shared(p);
}

__device__ inline void mbar_init(unsigned long long* bar, unsigned count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count)
               : "memory");
}

__device__ inline void mbar_expect_tx(unsigned long long* bar, unsigned bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)),
               "r"(bytes)
               : "memory");
}

__device__ inline bool mbar_try_wait(unsigned long long* bar, unsigned parity) {
  unsigned ok;
  asm volatile(
      "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n"
      " selp.u32 %0, 1, 0, p;\n}\n"
      : "=r"(ok)
      : "r"(smem_u32(bar)), "r"(parity)
      : "memory");
  return ok != 0;
}

// bounded wait: false when the budget ran out
__device__ inline bool mbar_wait(unsigned long long* bar, unsigned parity) {
  const long long t0 = clock64();
  while (!mbar_try_wait(bar, parity))
    if (clock64() - t0 > kWaitBudget) return false;
  return true;
}

__device__ inline void tma_load_4d(void* dst, const CUtensorMap* map, int x, int y, int z, int c,
                                   unsigned long long* bar) {
  asm volatile(
      "cp.async.bulk.tensor.4d.shared::cluster.global.tile.mbarrier::complete_tx::bytes"
      " [%0], [%1, {%2, %3, %4, %5}], [%6];" ::"r"(smem_u32(dst)),
      "l"((unsigned long long)map), "r"(x), "r"(y), "r"(z), "r"(c), "r"(smem_u32(bar))
      : "memory");
}

template <typename T, int TY>
struct TmaGeom {
  static constexpr int TX = 32;
  static constexpr int HP = 16 / (int)sizeof(T);  // x halo pad keeping boxes 16-byte aligned
  static constexpr int BXW = TX + 2 * HP;
  static constexpr int BYH = TY + 2;
  static constexpr int BOX = 3 * BYH * BXW;      // elements of one array's box
  static constexpr int BOXB = (BOX * (int)sizeof(T) + 127) / 128 * 128;
  static constexpr int BX = TX + 1, BY = TY + 1;
};

template <typename T, int TY, int NS>
constexpr size_t tma_smem_bytes() {
  using G = TmaGeom<T, TY>;
  return (size_t)NS * 3 * G::BOXB + 2 * 3 * G::BY * G::BX * sizeof(T) + NS * 8 + 128;
}

template <typename T, int TY, int NS>
__global__ void __launch_bounds__(32 * TY)
    k_fused_tma(const __grid_constant__ CUtensorMap tD, const __grid_constant__ CUtensorMap tI,
                const __grid_constant__ CUtensorMap tB, Mesh m, const T* __restrict__ Din,
                const T* __restrict__ Bin, const T* __restrict__ ie, T* __restrict__ Dout,
                T* __restrict__ Bout, T cB, T cD, int zchunk, unsigned int* err) {
  using G = TmaGeom<T, TY>;
  constexpr int TX = G::TX, HP = G::HP, BXW = G::BXW, BYH = G::BYH, BX = G::BX, BY = G::BY;
  constexpr int NT = TX * TY;
  extern __shared__ __align__(128) unsigned char smem[];
  unsigned char* base = (unsigned char*)(((size_t)smem + 127) & ~(size_t)127);
  T* sBp = (T*)(base + (size_t)NS * 3 * G::BOXB);  // [2][3][BY][BX]
  unsigned long long* bars =
      (unsigned long long*)((unsigned char*)sBp + 2 * 3 * BY * BX * sizeof(T));
  __shared__ int s_fail;

  const int nx = m.n[0], ny = m.n[1], nz = m.n[2];
  const int64_t V = m.V;
  const int64_t P = (int64_t)nx * ny;
  const int x0 = blockIdx.x * TX, y0 = blockIdx.y * TY;
  const int z0 = blockIdx.z * zchunk;
  const int z1 = min(z0 + zchunk, nz);
  const int R = (z1 - z0) + 2;  // planes z0-1 .. z1
  const int tid = threadIdx.y * TX + threadIdx.x;
  const int TXe = min(TX, nx - x0), TYe = min(TY, ny - y0);
  const bool edge = (x0 == 0) || (x0 + TXe == nx) || (y0 == 0) || (y0 + TYe == ny);
  constexpr unsigned kTx = 3u * G::BOX * sizeof(T);

  auto boxp = [&](int stage, int arr) -> T* {
    return (T*)(base + ((size_t)stage * 3 + arr) * G::BOXB);
  };
  auto wrapz = [&](int k) { return k >= nz ? k - nz : (k < 0 ? k + nz : k); };
  auto issue = [&](int r) {  // plane z0 - 1 + r into stage r % NS
    const int s = r % NS;
    const int z = wrapz(z0 - 1 + r);
    mbar_expect_tx(&bars[s], kTx);
    tma_load_4d(boxp(s, 0), &tD, x0 - HP, y0 - 1, z, 0, &bars[s]);
    tma_load_4d(boxp(s, 1), &tI, x0 - HP, y0 - 1, z, 0, &bars[s]);
    tma_load_4d(boxp(s, 2), &tB, x0 - HP, y0 - 1, z, 0, &bars[s]);
  };
  // the periodic halo ring of a boundary tile, from the opposite side
  auto patch = [&](int r) {
    const int s = r % NS;
    const int64_t pk = (int64_t)wrapz(z0 - 1 + r) * P;
    const int W = TXe + 2, H = TYe + 2;
    const int ring = 2 * W + 2 * (H - 2);
    for (int e = tid; e < ring; e += NT) {
      int iy, ixr;
      if (e < W) {
        iy = 0;
        ixr = e;
      } else if (e < 2 * W) {
        iy = H - 1;
        ixr = e - W;
      } else {
        const int t = e - 2 * W;
        iy = 1 + (t >> 1);
        ixr = (t & 1) ? W - 1 : 0;
      }
      const int ix = HP - 1 + ixr;
      int gx = x0 - HP + ix, gy = y0 - 1 + iy;
      if (gx >= 0 && gx < nx && gy >= 0 && gy < ny) continue;
      gx = gx < 0 ? gx + nx : (gx >= nx ? gx - nx : gx);
      gy = gy < 0 ? gy + ny : (gy >= ny ? gy - ny : gy);
      const int64_t v = pk + (int64_t)gy * nx + gx;
#pragma unroll
      for (int c = 0; c < 3; ++c) {
        const int o = (c * BYH + iy) * BXW + ix;
        boxp(s, 0)[o] = Din[c * V + v];
        boxp(s, 1)[o] = ie[c * V + v];
        boxp(s, 2)[o] = Bin[c * V + v];
      }
    }
  };
  auto E = [&](const T* d, const T* i, int c, int iy, int ix) -> T {
    const int o = (c * BYH + iy) * BXW + ix;
    return d[o] * i[o];
  };
  // B' on the tile and its low halo: element (bx, by) is site
  // (x0 - 1 + bx, y0 - 1 + by), box position (by, bx + HP - 1)
  auto compute_B = [&](int r, int slot, bool store, int64_t pk) {
    const T* dc = boxp(r % NS, 0);
    const T* ic = boxp(r % NS, 1);
    const T* bb = boxp(r % NS, 2);
    const T* dn = boxp((r + 1) % NS, 0);
    const T* in = boxp((r + 1) % NS, 1);
    T* sB = sBp + (size_t)slot * 3 * BY * BX;
    for (int e = tid; e < BX * BY; e += NT) {
      const int by = e / BX, bx = e - by * BX;
      const int iy = by, ix = bx + HP - 1;
      const T Ex = E(dc, ic, 0, iy, ix), Ey = E(dc, ic, 1, iy, ix), Ez = E(dc, ic, 2, iy, ix);
      const T Ey_x = E(dc, ic, 1, iy, ix + 1), Ez_x = E(dc, ic, 2, iy, ix + 1);
      const T Ex_y = E(dc, ic, 0, iy + 1, ix), Ez_y = E(dc, ic, 2, iy + 1, ix);
      const T Ex_z = E(dn, in, 0, iy, ix), Ey_z = E(dn, in, 1, iy, ix);
      const T bxv = bb[(0 * BYH + iy) * BXW + ix] - cB * (((Ey + Ez_y) - Ey_z) - Ez);
      const T byv = bb[(1 * BYH + iy) * BXW + ix] - cB * (((Ez + Ex_z) - Ez_x) - Ex);
      const T bzv = bb[(2 * BYH + iy) * BXW + ix] - cB * (((Ex + Ey_x) - Ex_y) - Ey);
      sB[(0 * BY + by) * BX + bx] = bxv;
      sB[(1 * BY + by) * BX + bx] = byv;
      sB[(2 * BY + by) * BX + bx] = bzv;
      if (store && bx >= 1 && by >= 1 && bx <= TXe && by <= TYe) {
        const int64_t v = pk + (int64_t)(y0 - 1 + by) * nx + (x0 - 1 + bx);
        Bout[v] = bxv;
        Bout[V + v] = byv;
        Bout[2 * V + v] = bzv;
      }
    }
  };
  // the kernel stops here on a failed wait: drain the copies in flight
  // (bounded) so no TMA write lands after the CTA exits
  auto bail = [&](int next_issue, int consumed) {
    if (tid == 0) {
      atomicOr(err, kErrTimeout);
      for (int r = consumed; r < next_issue; ++r)
        if (!mbar_wait(&bars[r % NS], (unsigned)((r / NS) & 1))) break;
    }
  };

  if (tid == 0) {
    s_fail = 0;
    for (int s = 0; s < NS; ++s) mbar_init(&bars[s], 1);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  __syncthreads();
  int issued = 0;
  if (tid == 0)
    for (; issued < NS && issued < R; ++issued) issue(issued);
  issued = min(NS, R);  // every thread tracks the count

  // prologue: planes r = 0 (z0 - 1) and r = 1 (z0), B' of z0 - 1
  if (!mbar_wait(&bars[0], 0) || !mbar_wait(&bars[1], 0)) s_fail = 1;
  if (edge) {
    patch(0);
    patch(1);
  }
  __syncthreads();
  if (s_fail) {
    bail(issued, 0);
    return;
  }
  compute_B(0, 0, false, 0);
  int bp = 0, bc = 1;
  for (int k = z0; k < z1; ++k) {
    const int r = k - z0 + 1;  // plane k; plane k + 1 is r + 1
    if (!mbar_wait(&bars[(r + 1) % NS], (unsigned)(((r + 1) / NS) & 1))) s_fail = 1;
    if (edge && !s_fail) patch(r + 1);
    __syncthreads();  // plane r+1 ready; plane r-1 and sB[bc] no longer read
    if (s_fail) {
      bail(issued, r);
      return;
    }
    if (issued < R) {
      if (tid == 0) {
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
        issue(issued);
      }
      ++issued;
    }
    const int64_t pk = (int64_t)k * P;
    compute_B(r, bc, true, pk);
    __syncthreads();
    const int tx = threadIdx.x, ty = threadIdx.y;
    if (tx < TXe && ty < TYe) {
      const T* dcur = boxp(r % NS, 0);
      const T* sB = sBp + (size_t)bc * 3 * BY * BX;
      const T* sP = sBp + (size_t)bp * 3 * BY * BX;
      const int bx = tx + 1, by = ty + 1;
      const int iy = ty + 1, ix = tx + HP;
      auto Bc = [&](int c, int yy, int xx) { return sB[(c * BY + yy) * BX + xx]; };
      const T Bx = Bc(0, by, bx), By = Bc(1, by, bx), Bz = Bc(2, by, bx);
      const int64_t v = pk + (int64_t)(y0 + ty) * nx + (x0 + tx);
      Dout[v] = dcur[(0 * BYH + iy) * BXW + ix] +
                cD * (((Bz - Bc(2, by - 1, bx)) - By) + sP[(1 * BY + by) * BX + bx]);
      Dout[V + v] = dcur[(1 * BYH + iy) * BXW + ix] +
                    cD * (((Bx - sP[(0 * BY + by) * BX + bx]) - Bz) + Bc(2, by, bx - 1));
      Dout[2 * V + v] = dcur[(2 * BYH + iy) * BXW + ix] +
                        cD * (((By - Bc(1, by, bx - 1)) - Bx) + Bc(0, by - 1, bx));
    }
    bp ^= 1;
    bc ^= 1;
  }
}

PFN_cuTensorMapEncodeTiled_v12000 encoder() {
  static PFN_cuTensorMapEncodeTiled_v12000 fn = nullptr;
  static bool tried = false;
  if (!tried) {
    tried = true;
    void* p = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault,
                                         &q) == cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      fn = (PFN_cuTensorMapEncodeTiled_v12000)p;
    cudaGetLastError();
  }
  return fn;
}

template <typename T, int TY, int NS>
void launch_t(const Mesh& m, const TmaMaps& maps, int par, const void* Din, const void* Bin,
              const void* ie, void* Dout, void* Bout, double cB, double cD, int zchunk,
              unsigned int* err, cudaStream_t st) {
  constexpr size_t smem = tma_smem_bytes<T, TY, NS>();
  static bool attr = false;
  if (!attr) {
    cudaFuncSetAttribute(k_fused_tma<T, TY, NS>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                         (int)smem);
    attr = true;
  }
  const dim3 grid((m.n[0] + 31) / 32, (m.n[1] + TY - 1) / TY, (m.n[2] + zchunk - 1) / zchunk);
  const int mi = TmaMaps::index(TY);
  k_fused_tma<T, TY, NS><<<grid, dim3(32, TY, 1), smem, st>>>(
      maps.D[par][mi], maps.ie[mi], maps.B[par][mi], m, (const T*)Din, (const T*)Bin,
      (const T*)ie, (T*)Dout, (T*)Bout, (T)cB, (T)cD, zchunk, err);
}

}  // namespace

bool tma_supported(const Mesh& m, int prec) {
  const int es = prec == 1 ? 4 : 8;
  if (((int64_t)m.n[0] * es) % 16 != 0) return false;
  return encoder() != nullptr;
}

// One 4-D map (x, y, z, component) per array and tile height.
bool tma_make_maps(const Mesh& m, int prec, void* const D[2], void* const B[2], void* ie,
                   TmaMaps* out) {
  PFN_cuTensorMapEncodeTiled_v12000 enc = encoder();
  if (!enc || !tma_supported(m, prec)) return false;
  const int es = prec == 1 ? 4 : 8;
  const int HP = 16 / es;
  const CUtensorMapDataType dt =
      prec == 1 ? CU_TENSOR_MAP_DATA_TYPE_FLOAT32 : CU_TENSOR_MAP_DATA_TYPE_FLOAT64;
  const cuuint64_t dims[4] = {(cuuint64_t)m.n[0], (cuuint64_t)m.n[1], (cuuint64_t)m.n[2], 3};
  const cuuint64_t strides[3] = {(cuuint64_t)m.n[0] * es, (cuuint64_t)m.n[0] * m.n[1] * es,
                                 (cuuint64_t)m.V * es};
  const cuuint32_t estr[4] = {1, 1, 1, 1};
  for (int t = 0; t < 3; ++t) {
    const int TY = TmaMaps::ty(t);
    const cuuint32_t box[4] = {(cuuint32_t)(32 + 2 * HP), (cuuint32_t)(TY + 2), 1, 3};
    auto mk = [&](CUtensorMap* map, void* ptr) {
      return enc(map, dt, 4, ptr, dims, strides, box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE,
                 CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                 CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
    };
    for (int p = 0; p < 2; ++p)
      if (!mk(&out->D[p][t], D[p]) || !mk(&out->B[p][t], B[p])) return false;
    if (!mk(&out->ie[t], ie)) return false;
  }
  return true;
}

void launch_fused_tma(const Mesh& m, int prec, const TmaMaps& maps, int par, const void* Din,
                      const void* Bin, const void* ie, void* Dout, void* Bout, double cB,
                      double cD, FusedCfg cfg, unsigned int* err, cudaStream_t st) {
  if (cfg.zchunk < 1) cfg.zchunk = 8;
  if (cfg.zchunk > m.n[2]) cfg.zchunk = m.n[2];
  if (prec == 1) {
    switch (cfg.ty) {
      case 4: launch_t<float, 4, 4>(m, maps, par, Din, Bin, ie, Dout, Bout, cB, cD, cfg.zchunk, err, st); break;
      case 16: launch_t<float, 16, 3>(m, maps, par, Din, Bin, ie, Dout, Bout, cB, cD, cfg.zchunk, err, st); break;
      default: launch_t<float, 8, 4>(m, maps, par, Din, Bin, ie, Dout, Bout, cB, cD, cfg.zchunk, err, st);
    }
  } else {
    switch (cfg.ty) {
      case 4: launch_t<double, 4, 4>(m, maps, par, Din, Bin, ie, Dout, Bout, cB, cD, cfg.zchunk, err, st); break;
      case 16: launch_t<double, 16, 3>(m, maps, par, Din, Bin, ie, Dout, Bout, cB, cD, cfg.zchunk, err, st); break;
      default: launch_t<double, 8, 3>(m, maps, par, Din, Bin, ie, Dout, Bout, cB, cD, cfg.zchunk, err, st);
    }
  }
}

}  // namespace memd
