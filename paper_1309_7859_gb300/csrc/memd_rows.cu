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
#include "memd_rows.cuh"

namespace memd {

namespace {

using rows::rows_segment;

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
