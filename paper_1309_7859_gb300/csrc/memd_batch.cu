// memd_batch.cu -- many independent MEMD systems stepped together.
//
// A batch holds a device table of replica descriptors (mesh, step
// parameters, field and particle pointers) and two CTA->replica maps, one
// for the field tiles and one for the particle quads.  Each time step is one
// CUDA graph of four launches covering every member: the charge transfer of
// the drift on a side stream beside the fused field update, then the
// transfer application, then the force gather, which also closes each
// replica's step.  Small systems that would each leave most SMs idle fill
// the GPU together, and the per-step launch cost is paid once for all.
#include <algorithm>
#include <cstring>
#include <string>
#include <vector>

#include "memd.h"
#include "memd_ctx.cuh"
#include "memd_internal.cuh"

using namespace memd;

struct memd_batch {
  std::vector<memd_ctx*> m;
  std::vector<int> gen;    // member generations the tables were built for
  std::vector<int> base;   // member parity when the batch parity was 0
  int bpar = 0;            // batch parity
  int prec = 0;
  int device = 0;
  cudaStream_t stream = nullptr;
  cudaStream_t side = nullptr;
  cudaEvent_t fork = nullptr, join = nullptr, ev0 = nullptr, ev1 = nullptr;
  // memd_batch_step_io's one-step graph (per buffer parity) and its events
  cudaGraphExec_t io_graph[2] = {nullptr, nullptr};
  cudaEvent_t io_dep = nullptr, io_join = nullptr;
  cudaEvent_t evp[6] = {nullptr, nullptr, nullptr, nullptr, nullptr, nullptr};  // phases
  RepDesc* d_desc = nullptr;
  int* d_field_rep = nullptr;
  int* d_part_rep = nullptr;
  int* d_part_rep_w = nullptr;  // CTA -> replica of the one-thread-per-charge kernels
  int n_field = 0, n_part = 0, n_part_w = 0;
  bool wide = false;            // deposition and gather one thread per charge
  double field_bytes = 0.0;
  int f_ty = kBatchTY, f_pf = kBatchPF32, f_z = kBatchZ;  // field tiles (autotuned)
  int f_w = 32;                                          // tile width: 32 or 16 sites
  int f_rows = 0;         // 0: site tiles; nt > 0: the row kernel, nt threads a CTA
  int f_kind = MEMD_FIELD_AUTO;  // the kernel family asked for at create
  RowSeg* d_segs = nullptr;
  int* d_seg_first = nullptr;
  int n_rows_ctas = 0;
  // transfer application: dense pass over (replica, chunk) pairs, or the
  // sparse per-charge form (MEMD_APPLY_* of member 0; AUTO is sparse)
  bool apply_dense = false;
  int2* d_apply_chunk = nullptr;
  int n_apply_chunk = 0;
  cudaGraphExec_t graph[2] = {nullptr, nullptr};
  // single-launch step (k_batch_step): the engine asked for, whether it runs,
  // its grid, the CTAs that start with field work, planes per field item, the
  // four work queues and the scheduling state
  int engine = MEMD_STEP_AUTO;
  bool single = false;
  bool single_graph_ok = true;  // its launch can be captured in a graph
  bool overlap = true;  // graph engine: the deposition beside the field pass
  int bs_grid = 0;
  int bs_field_ctas = -1;   // -1: half the grid
  int bs_item_planes = 0;   // 0: chosen from the work (about one item per CTA)
  BatchItem* d_q[2] = {nullptr, nullptr};
  int nq[2] = {0, 0};
  BatchSched* d_sched = nullptr;
  RepSync* d_sync = nullptr;
  // memd_batch_step_io: the members' particle offsets (host and device) and
  // the I/O block (page-locked host memory and its device mirror)
  std::vector<int64_t> ioff;
  int64_t* d_ioff = nullptr;
  unsigned char* io_host = nullptr;
  void* io_dev = nullptr;
  int64_t io_ntot = -1;
  int timing = -1;  // -1: time the field update when member 0 does; 0 / 1: off / on
  int g_thermo = -1;
  double g_gamma = 0.0, g_kT = 0.0;
  bool timing_pending = false;
  double field_ms = 0.0;
  double phase_ms[3] = {0.0, 0.0, 0.0};  // deposition, transfer application, gather
  long long field_launches = 0;
  std::string last_error;
  // the batch's own tables come from member 0's allocator but are tracked
  // here, so members may be destroyed after the batch without double frees
  memd_alloc_fn alloc = nullptr;
  memd_free_fn free_fn = nullptr;
  void* alloc_user = nullptr;
  std::vector<std::pair<void*, size_t>> blocks;
};

namespace {

memd_status bfail(memd_batch* b, memd_status s, const std::string& why) {
  if (b) b->last_error = why;
  return s;
}

#define BCK(call)                                                                    \
  do {                                                                               \
    cudaError_t e_ = (call);                                                         \
    if (e_ != cudaSuccess)                                                           \
      return bfail(b, MEMD_ERR_CUDA, std::string(#call) + ": " + cudaGetErrorString(e_)); \
  } while (0)

void drop(memd_batch* b) {
  for (cudaGraphExec_t& g : b->graph)
    if (g) {
      cudaGraphExecDestroy(g);
      g = nullptr;
    }
  for (cudaGraphExec_t& g : b->io_graph)
    if (g) {
      cudaGraphExecDestroy(g);
      g = nullptr;
    }
}

void* balloc(memd_batch* b, size_t bytes) {
  if (bytes < 256) bytes = 256;
  void* p = nullptr;
  if (b->alloc) {
    p = b->alloc(b->alloc_user, bytes, (void*)b->stream);
  } else if (cudaMalloc(&p, bytes) != cudaSuccess) {
    cudaGetLastError();
    p = nullptr;
  }
  if (p) b->blocks.emplace_back(p, bytes);
  return p;
}

void free_tables(memd_batch* b) {
  for (auto& blk : b->blocks) {
    if (b->free_fn)
      b->free_fn(b->alloc_user, blk.first, blk.second, (void*)b->stream);
    else
      cudaFree(blk.first);
  }
  b->blocks.clear();
  b->d_desc = nullptr;
  b->d_field_rep = b->d_part_rep = b->d_part_rep_w = nullptr;
  b->d_segs = nullptr;
  b->d_seg_first = nullptr;
  b->n_rows_ctas = 0;
  b->d_apply_chunk = nullptr;
  b->n_apply_chunk = 0;
  b->d_ioff = nullptr;
  for (int q = 0; q < 2; ++q) {
    b->d_q[q] = nullptr;
    b->nq[q] = 0;
  }
  b->d_sched = nullptr;
  b->d_sync = nullptr;
  b->single = false;
}

// Work items of the single-launch step.  Field: each member's row tiles (the
// row kernel's geometry for kBatchStepThreads threads) cut into ranges of at
// most `planes` planes; particles: chunks of kBatchStepThreads / 4 charges,
// kBatchChunksPerItem a particle item, at least one item per member (its last
// gather item closes the member's step); the deposition items go in a queue,
// the application and gather items are counted per member.  False when a
// member does not fit the row tiles.
bool batch_items(memd_batch* b, std::vector<RepDesc>& desc, int grid,
                 std::vector<BatchItem> (&q)[2]) {
  const int W = rows_sites_per_thread(b->prec);
  const int nt = kBatchStepThreads;
  struct Tile {
    int rep, y0, rows, nz;
  };
  std::vector<Tile> tiles;
  long long tile_planes = 0;
  for (size_t r = 0; r < b->m.size(); ++r) {
    const memd_ctx* c = b->m[r];
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
      tiles.push_back(Tile{(int)r, y0, std::min(Rt, ny - y0), nz});
      tile_planes += nz;
    }
  }
  int planes = b->bs_item_planes;
  if (planes <= 0) planes = std::max<long long>(8, (tile_planes + grid - 1) / grid);
  for (auto& v : q) v.clear();
  for (size_t r = 0; r < b->m.size(); ++r) {
    desc[r].b_nf = 0;
    for (const Tile& t : tiles) {
      if (t.rep != (int)r) continue;
      const int nseg = (t.nz + planes - 1) / planes;
      for (int k = 0; k < nseg; ++k) {
        const int za = (int)((int64_t)t.nz * k / nseg), zb = (int)((int64_t)t.nz * (k + 1) / nseg);
        q[kItemField].push_back(BatchItem{(int)r, t.y0, t.rows, za, zb});
        desc[r].b_nf += 1;
      }
    }
    const int nc = (int)std::max<int64_t>(1, (4 * b->m[r]->P.n + nt - 1) / nt);
    const int np = (nc + kBatchChunksPerItem - 1) / kBatchChunksPerItem;
    desc[r].b_nc = nc;
    desc[r].b_np = np;
    for (int k = 0; k < np; ++k) q[kItemDeposit].push_back(BatchItem{(int)r, k, 0, 0, 0});
  }
  return true;
}

void free_io(memd_batch* b) {
  for (cudaGraphExec_t& g : b->io_graph)  // they hold the block's addresses
    if (g) {
      cudaGraphExecDestroy(g);
      g = nullptr;
    }
  if (b->io_host) cudaFreeHost(b->io_host);
  b->io_host = nullptr;
  if (b->io_dev) {
    if (b->free_fn)
      b->free_fn(b->alloc_user, b->io_dev, (size_t)batch_io_bytes(b->io_ntot, (int)b->m.size()),
                 (void*)b->stream);
    else
      cudaFree(b->io_dev);
  }
  b->io_dev = nullptr;
  b->io_ntot = -1;
}

// Work of the row kernel: every replica's planes cut into full-width tiles
// of at most nt / (nx / W) - 2 rows (one halo row on either side), each
// tile-plane weighted by its cost (below); the weighted list is split
// into nctas contiguous ranges of equal weight, one per CTA of a persistent
// grid, each range a list of segments.  False when a replica does not fit
// (x extent not a multiple of the vector width, rows too wide for nt, or a
// field buffer not 16-byte aligned).
// (Re)build the descriptor table and the CTA maps from the members' state;
// the batch parity restarts at 0 with each member's current buffer first.
memd_status build_tables(memd_batch* b, bool sync = true) {
  drop(b);
  free_tables(b);
  const int R = (int)b->m.size();
  std::vector<RepDesc> desc(R);
  std::vector<int> frep, prep, pwrep;
  std::vector<int2> achunk;
  b->field_bytes = 0.0;
  for (int r = 0; r < R; ++r) {
    memd_ctx* c = b->m[r];
    {
      // transfers a member's single-launch steps left pending go in first
      const memd_status fe = memd_flush(c);
      if (fe != MEMD_OK) return bfail(b, fe, "member flush");
    }
    RepDesc& d = desc[r];
    std::memset(&d, 0, sizeof(d));
    d.m = c->mesh;
    d.sp = memd_step_params(c, 0, 0.0, 0.0);
    d.P = c->P;
    for (int k = 0; k < 2; ++k) {
      d.D[k] = c->Dbuf[(c->cur + k) & 1];
      d.B[k] = c->Bbuf[(c->cur + k) & 1];
    }
    d.ie = c->ie;
    d.ie64 = c->ie64;
    d.Lg = c->Lg;
    d.Tb = c->Tb;
    d.ds = c->ds;
    d.f_tx = (c->mesh.n[0] + b->f_w - 1) / b->f_w;
    d.f_ty = (c->mesh.n[1] + b->f_ty - 1) / b->f_ty;
    d.f_zchunk = std::min(c->mesh.n[2], b->f_z);
    const int nzc = (c->mesh.n[2] + d.f_zchunk - 1) / d.f_zchunk;
    d.f_first = (int)frep.size();
    for (int t = 0; t < d.f_tx * d.f_ty * nzc; ++t) frep.push_back(r);
    d.p_first = (int)prep.size();
    d.p_ctas = (int)std::max<int64_t>(1, (4 * c->P.n + kBatchQuadThreads - 1) / kBatchQuadThreads);
    for (int t = 0; t < d.p_ctas; ++t) prep.push_back(r);
    d.pw_first = (int)pwrep.size();
    d.pw_ctas = (int)std::max<int64_t>(1, (c->P.n + kWideThreads - 1) / kWideThreads);
    for (int t = 0; t < d.pw_ctas; ++t) pwrep.push_back(r);
    const int64_t nch = (3 * c->mesh.V + kApplyChunk - 1) / kApplyChunk;
    for (int64_t k = 0; k < nch; ++k) achunk.push_back(make_int2(r, (int)k));
    b->base[r] = c->cur;
    b->gen[r] = c->gen;
    b->field_bytes += 15.0 * (double)memd_esz(c) * (double)c->mesh.V;
  }
  b->ioff.assign(R + 1, 0);
  for (int r = 0; r < R; ++r) b->ioff[r + 1] = b->ioff[r] + b->m[r]->P.n;
  b->wide = b->ioff[R] >= kWideMinCharges;
  b->n_part_w = (int)pwrep.size();
  // the single-launch step when asked for and it can run: cooperative
  // launches, a resident grid of its CTAs, and every member in row tiles
  std::vector<BatchItem> items[2];
  if (b->engine == MEMD_STEP_SINGLE) {
    int coop = 0, sms = 0;
    BCK(cudaDeviceGetAttribute(&coop, cudaDevAttrCooperativeLaunch, b->device));
    BCK(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, b->device));
    const int occ = coop ? batch_step_occupancy(b->prec) : 0;
    b->bs_grid = occ * sms;
    b->single = b->bs_grid > 0 && batch_items(b, desc, b->bs_grid, items);
  }
  b->bpar = 0;
  b->n_field = (int)frep.size();
  b->n_part = (int)prep.size();
  b->d_desc = (RepDesc*)balloc(b, sizeof(RepDesc) * R);
  b->d_field_rep = (int*)balloc(b, sizeof(int) * std::max(1, b->n_field));
  b->d_part_rep = (int*)balloc(b, sizeof(int) * std::max(1, b->n_part));
  b->d_ioff = (int64_t*)balloc(b, sizeof(int64_t) * (R + 1));
  b->d_part_rep_w = (int*)balloc(b, sizeof(int) * std::max(1, b->n_part_w));
  if (!b->d_desc || !b->d_field_rep || !b->d_part_rep || !b->d_ioff || !b->d_part_rep_w)
    return bfail(b, MEMD_ERR_OOM, "batch tables");
  BCK(cudaMemcpyAsync(b->d_part_rep_w, pwrep.data(), sizeof(int) * b->n_part_w,
                      cudaMemcpyHostToDevice, b->stream));
  BCK(cudaMemcpyAsync(b->d_ioff, b->ioff.data(), sizeof(int64_t) * (R + 1),
                      cudaMemcpyHostToDevice, b->stream));
  BCK(cudaMemcpyAsync(b->d_desc, desc.data(), sizeof(RepDesc) * R, cudaMemcpyHostToDevice,
                      b->stream));
  BCK(cudaMemcpyAsync(b->d_field_rep, frep.data(), sizeof(int) * b->n_field,
                      cudaMemcpyHostToDevice, b->stream));
  BCK(cudaMemcpyAsync(b->d_part_rep, prep.data(), sizeof(int) * b->n_part,
                      cudaMemcpyHostToDevice, b->stream));
  if (b->single) {
    for (int q = 0; q < 2; ++q) {
      b->nq[q] = (int)items[q].size();
      b->d_q[q] = (BatchItem*)balloc(b, sizeof(BatchItem) * std::max<size_t>(1, items[q].size()));
      if (!b->d_q[q]) return bfail(b, MEMD_ERR_OOM, "batch work queues");
      BCK(cudaMemcpyAsync(b->d_q[q], items[q].data(), sizeof(BatchItem) * items[q].size(),
                          cudaMemcpyHostToDevice, b->stream));
    }
    b->d_sched = (BatchSched*)balloc(b, sizeof(BatchSched));
    b->d_sync = (RepSync*)balloc(b, sizeof(RepSync) * R);
    if (!b->d_sched || !b->d_sync) return bfail(b, MEMD_ERR_OOM, "batch scheduling state");
    BCK(cudaMemsetAsync(b->d_sched, 0, sizeof(BatchSched), b->stream));
    BCK(cudaMemsetAsync(b->d_sync, 0, sizeof(RepSync) * R, b->stream));
  }
  b->apply_dense = apply_dense(b->m[0]->apply_mode);
  if (b->apply_dense) {
    b->n_apply_chunk = (int)achunk.size();
    b->d_apply_chunk = (int2*)balloc(b, sizeof(int2) * std::max(1, b->n_apply_chunk));
    if (!b->d_apply_chunk) return bfail(b, MEMD_ERR_OOM, "batch apply table");
    BCK(cudaMemcpyAsync(b->d_apply_chunk, achunk.data(), sizeof(int2) * b->n_apply_chunk,
                        cudaMemcpyHostToDevice, b->stream));
  }
  if (b->f_rows > 0) {
    int sms = 0;
    BCK(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, b->device));
    const int occ = rows_occupancy(b->prec, b->f_rows);
    std::vector<RowSeg> segs;
    std::vector<int> first;
    if (occ > 0 && rows_plan(b->m, b->prec, b->f_rows, occ * sms, segs, first)) {
      b->n_rows_ctas = occ * sms;
      b->d_segs = (RowSeg*)balloc(b, sizeof(RowSeg) * std::max<size_t>(1, segs.size()));
      b->d_seg_first = (int*)balloc(b, sizeof(int) * first.size());
      if (!b->d_segs || !b->d_seg_first) return bfail(b, MEMD_ERR_OOM, "batch row tables");
      BCK(cudaMemcpyAsync(b->d_segs, segs.data(), sizeof(RowSeg) * segs.size(),
                          cudaMemcpyHostToDevice, b->stream));
      BCK(cudaMemcpyAsync(b->d_seg_first, first.data(), sizeof(int) * first.size(),
                          cudaMemcpyHostToDevice, b->stream));
    } else {
      b->f_rows = 0;  // some member does not fit the row kernel: site tiles
    }
  }
  // the host tables were staged by the copies above, so they may go; a
  // caller that queues more work on the stream need not wait
  if (sync) BCK(cudaStreamSynchronize(b->stream));
  return MEMD_OK;
}

// the batch's field update: row kernel or site tiles
cudaError_t launch_field(memd_batch* b, int par, cudaStream_t st) {
  if (b->f_rows > 0)
    return launch_rows_batch(b->prec, b->d_desc, b->d_segs, b->d_seg_first, b->n_rows_ctas,
                             b->f_rows, par, st);
  launch_fused_batch(b->prec, b->d_desc, b->d_field_rep, b->n_field, par, b->f_ty, b->f_pf,
                     b->f_w, st);
  return cudaGetLastError();
}

// Reads a scratch buffer larger than L2, leaving L2 full of clean lines of
// it: the field update timed next starts from DRAM, as in a step.
__global__ void k_read_flush(const float4* __restrict__ p, size_t n4, float* sink) {
  float acc = 0.f;
  for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n4;
       i += (size_t)gridDim.x * blockDim.x) {
    const float4 v = p[i];
    acc += v.x + v.y + v.z + v.w;
  }
  if (acc == 1234.5f) *sink = acc;  // keeps the loads
}

// Field tiles of the batched kernel: tile width 32 or 16 sites, height 4, 8
// or (FP32) 16 rows, loads 1 or 2 planes ahead, 4 to 32 planes per CTA, timed on the members' buffers (the
// update reads the current parity and writes the other one, which the next
// step overwrites with the same values).  Each sample is one launch after
// a 256 MiB read that evicts L2; median of 3 samples after a warm-up.
memd_status autotune_batch(memd_batch* b) {
  memd::NvtxRange nvtx_("autotune_batch");
  static const int tys[3] = {4, 8, 16}, zs[4] = {4, 8, 16, 32};
  const int nty = b->prec == MEMD_FP32 ? 3 : 2;  // FP64 16-row tiles exceed static shared memory
  const int pfs = b->prec == MEMD_FP32 ? 2 : 1;  // FP64: one plane ahead (registers)
  cudaEvent_t e0, e1;
  BCK(cudaEventCreate(&e0));
  if (cudaEventCreate(&e1) != cudaSuccess) {
    cudaEventDestroy(e0);
    return bfail(b, MEMD_ERR_CUDA, "events");
  }
  const size_t flush_bytes = size_t(256) << 20;
  void* flush = nullptr;
  if (b->alloc) {
    flush = b->alloc(b->alloc_user, flush_bytes, (void*)b->stream);
  } else if (cudaMalloc(&flush, flush_bytes) != cudaSuccess) {
    cudaGetLastError();
    flush = nullptr;
  }
  if (!flush) {  // no room to tune: keep the defaults
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    return build_tables(b);
  }
  cudaMemsetAsync(flush, 0, flush_bytes, b->stream);
  float best = 1e30f;
  int bt = b->f_ty, bpf = b->f_pf, bz = b->f_z, bw = b->f_w, brows = 0;
  memd_status s = MEMD_OK;
  // one candidate: tables for it, a warm-up launch, then the median of three
  // launches each after an L2-evicting read
  auto sample = [&]() {
    s = build_tables(b);
    if (s != MEMD_OK) return;
    launch_field(b, 0, b->stream);
    float t[3];
    for (int r = 0; r < 3; ++r) {
      k_read_flush<<<4 * 152, 512, 0, b->stream>>>((const float4*)flush, flush_bytes / 16,
                                                    (float*)flush);
      cudaEventRecord(e0, b->stream);
      launch_field(b, 0, b->stream);
      cudaEventRecord(e1, b->stream);
      cudaEventSynchronize(e1);
      cudaEventElapsedTime(&t[r], e0, e1);
    }
    if (cudaGetLastError() != cudaSuccess) {
      s = bfail(b, MEMD_ERR_CUDA, "batch field autotune");
      return;
    }
    const float med = std::max(std::min(t[0], t[1]), std::min(std::max(t[0], t[1]), t[2]));
    if (med < best) {
      best = med;
      bt = b->f_ty;
      bpf = b->f_pf;
      bz = b->f_z;
      bw = b->f_w;
      brows = b->f_rows;
    }
  };
  if (b->f_kind != MEMD_FIELD_ROWS)
    for (int w = 32; w >= 16 && s == MEMD_OK; w /= 2)
      for (int a = 0; a < nty && s == MEMD_OK; ++a)
        for (int pf = 1; pf <= pfs && s == MEMD_OK; ++pf)
          for (int zi = 0; zi < 4 && s == MEMD_OK; ++zi) {
            b->f_rows = 0;
            b->f_w = w;
            b->f_ty = tys[a];
            b->f_pf = pf;
            b->f_z = zs[zi];
            sample();
          }
  if (b->f_kind != MEMD_FIELD_SITE)
    for (int nt = 256; nt <= 512 && s == MEMD_OK; nt *= 2) {
      b->f_rows = nt;
      sample();  // falls back to site tiles (f_rows = 0) when a member does not fit
    }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  cudaStreamSynchronize(b->stream);
  if (b->free_fn)
    b->free_fn(b->alloc_user, flush, flush_bytes, (void*)b->stream);
  else
    cudaFree(flush);
  if (s != MEMD_OK) return s;
  b->f_ty = bt;
  b->f_pf = bpf;
  b->f_z = bz;
  b->f_w = bw;
  b->f_rows = brows;
  return build_tables(b);
}

// The force gather that closes the step of buffer parity par (it reads the
// D that step wrote), for every replica.
cudaError_t gather_batch(memd_batch* b, int par, int thermo, double gamma, double kT,
                         cudaStream_t s) {
  if (b->wide)
    launch_gather_batch_wide(b->prec, b->d_desc, b->d_part_rep_w, b->n_part_w, par, thermo, s);
  else
    launch_gather_batch(b->prec, b->d_desc, b->d_part_rep, b->n_part, par, thermo, gamma, kT, s);
  return cudaGetLastError();
}

// the kick, drift and charge transfer of every replica
void deposit_batch(memd_batch* b, int thermo, double gamma, double kT, cudaStream_t s) {
  if (b->wide)
    launch_deposit_batch_wide(b->d_desc, b->d_part_rep_w, b->n_part_w, s);
  else
    launch_deposit_batch(b->d_desc, b->d_part_rep, b->n_part, thermo, gamma, kT, s);
}

// the step's transfers into the ledgers and the new D of every replica
void apply_batch(memd_batch* b, int par, cudaStream_t s) {
  if (b->apply_dense)
    launch_apply_dense_batch(b->prec, b->d_desc, b->d_apply_chunk, b->n_apply_chunk, par, s);
  else
    launch_apply_batch(b->prec, b->d_desc, b->d_part_rep, b->n_part, par, s);
}

bool batch_timed(const memd_batch* b) {
  return b->timing >= 0 ? b->timing != 0 : b->m[0]->time_kernels != 0;
}

// a new thermostat: the step graphs go, and every member's per-particle
// Langevin amplitudes are computed for it
void set_thermostat(memd_batch* b, int thermo, double gamma, double kT) {
  if (b->g_thermo == thermo && b->g_gamma == gamma && b->g_kT == kT) return;
  drop(b);
  for (memd_ctx* c : b->m) {
    launch_particle_constants(memd_step_params(c, thermo, gamma, kT), c->P, b->stream);
    c->sig_ready = false;  // a member stepped alone recomputes its own
  }
  b->g_thermo = thermo;
  b->g_gamma = gamma;
  b->g_kT = kT;
}

memd_status record(memd_batch* b, int par, int thermo, double gamma, double kT, bool timed) {
  const cudaStream_t st = b->stream;
  if (b->single) {
    // the whole step in one cooperative launch; with timing on, the event
    // pair brackets that launch
    BatchStepArgs a{};
    a.desc = b->d_desc;
    a.nrep = (int)b->m.size();
    for (int q = 0; q < 2; ++q) {
      a.q[q] = b->d_q[q];
      a.n[q] = b->nq[q];
    }
    a.sched = b->d_sched;
    a.sync = b->d_sync;
    a.par = par;
    a.thermo = thermo;
    a.gamma = gamma;
    a.kT = kT;
    a.field_ctas = b->bs_field_ctas >= 0 ? std::min(b->bs_field_ctas, b->bs_grid) : b->bs_grid / 2;
    a.wait_ns = 500000000ull;
    if (timed) BCK(cudaEventRecordWithFlags(b->ev0, st, cudaEventRecordExternal));
    BCK(launch_batch_step(b->prec, a, b->bs_grid, st));
    if (timed) {
      BCK(cudaEventRecordWithFlags(b->ev1, st, cudaEventRecordExternal));
      for (int k = 0; k < 6; ++k) BCK(cudaEventRecordWithFlags(b->evp[k], st, cudaEventRecordExternal));
    }
    return MEMD_OK;
  }
  auto deposit = [&](cudaStream_t s) { deposit_batch(b, thermo, gamma, kT, s); };
  auto apply = [&](cudaStream_t s) { apply_batch(b, par, s); };
  if (timed) {
    // instrumented: the four launches in turn on one stream, each between
    // its event pair, so that no launch's time holds another's
    BCK(cudaEventRecordWithFlags(b->ev0, st, cudaEventRecordExternal));
    BCK(launch_field(b, par, st));
    BCK(cudaEventRecordWithFlags(b->ev1, st, cudaEventRecordExternal));
    BCK(cudaEventRecordWithFlags(b->evp[0], st, cudaEventRecordExternal));
    deposit(st);
    BCK(cudaEventRecordWithFlags(b->evp[1], st, cudaEventRecordExternal));
    BCK(cudaEventRecordWithFlags(b->evp[2], st, cudaEventRecordExternal));
    apply(st);
    BCK(cudaEventRecordWithFlags(b->evp[3], st, cudaEventRecordExternal));
    BCK(cudaEventRecordWithFlags(b->evp[4], st, cudaEventRecordExternal));
    BCK(gather_batch(b, par, thermo, gamma, kT, st));
    BCK(cudaEventRecordWithFlags(b->evp[5], st, cudaEventRecordExternal));
    BCK(cudaGetLastError());
    return MEMD_OK;
  }
  // The deposition runs beside the field pass (neither reads what the other
  // writes): it is latency bound, the pass bandwidth bound, and the pass's
  // evict_first accesses leave the deposition's evict_last transfer words in
  // L2 for the application (64 replicas: 113.9 -> 109.8 us a step against
  // the two in turn).  Moving the gather that closes a step beside the next
  // field pass, ahead of the deposition, was slower (116.9 us): the two
  // particle kernels in turn then outlast the pass.  Without overlap (the
  // request server, whose admission work runs on other streams meanwhile)
  // the two run in turn.
  if (b->overlap) {
    BCK(cudaEventRecord(b->fork, st));
    BCK(cudaStreamWaitEvent(b->side, b->fork, 0));
    deposit(b->side);
    BCK(cudaEventRecord(b->join, b->side));
    BCK(launch_field(b, par, st));
    BCK(cudaStreamWaitEvent(st, b->join, 0));
  } else {
    BCK(launch_field(b, par, st));
    deposit(st);
  }
  apply(st);
  BCK(gather_batch(b, par, thermo, gamma, kT, st));
  BCK(cudaGetLastError());
  return MEMD_OK;
}

// One step of memd_batch_step_io with its copies.  The inputs' copy, their
// unpacking and the deposition run on the side stream beside the field pass
// (which reads no particle data); once the deposition is done, the moved part
// of the block (positions and image counters, final after the drift) is
// packed and copied back there beside the application and gather; the rest
// (velocities, forces, error words) after the gather.  The same kernels in
// the same order for every word as the copies around a step of the graph.
memd_status record_io(memd_batch* b, int par, int thermo, double gamma, double kT) {
  const cudaStream_t st = b->stream, sd = b->side;
  const int R = (int)b->m.size();
  const int64_t ntot = b->io_ntot;
  const IoLayout L = io_layout(ntot);
  const int64_t bytes = batch_io_bytes(ntot, R);
  unsigned char* dev = (unsigned char*)b->io_dev;
  BCK(cudaEventRecord(b->fork, st));
  BCK(cudaStreamWaitEvent(sd, b->fork, 0));
  BCK(cudaMemcpyAsync(dev, b->io_host, (size_t)L.f, cudaMemcpyHostToDevice, sd));
  launch_io_unpack_batch(b->d_desc, b->d_ioff, R, ntot, dev, sd);
  deposit_batch(b, thermo, gamma, kT, sd);
  BCK(cudaEventRecord(b->io_dep, sd));
  launch_io_pack_batch(b->d_desc, b->d_ioff, R, ntot, dev, sd, kIoMoved);
  BCK(cudaMemcpyAsync(b->io_host, dev, (size_t)L.vel, cudaMemcpyDeviceToHost, sd));
  BCK(cudaEventRecord(b->io_join, sd));
  BCK(launch_field(b, par, st));
  BCK(cudaStreamWaitEvent(st, b->io_dep, 0));
  apply_batch(b, par, st);
  BCK(gather_batch(b, par, thermo, gamma, kT, st));
  launch_io_pack_batch(b->d_desc, b->d_ioff, R, ntot, dev, st, kIoRest);
  BCK(cudaMemcpyAsync(b->io_host + L.vel, dev + L.vel, (size_t)(bytes - L.vel),
                      cudaMemcpyDeviceToHost, st));
  BCK(cudaStreamWaitEvent(st, b->io_join, 0));
  BCK(cudaGetLastError());
  return MEMD_OK;
}

void harvest(memd_batch* b) {
  if (!b->timing_pending) return;
  float ms = 0;
  if (cudaEventSynchronize(b->evp[5]) == cudaSuccess &&
      cudaEventElapsedTime(&ms, b->ev0, b->ev1) == cudaSuccess) {
    b->field_ms += ms;
    b->field_launches += 1;
    for (int k = 0; k < 3; ++k)
      if (cudaEventElapsedTime(&ms, b->evp[2 * k], b->evp[2 * k + 1]) == cudaSuccess)
        b->phase_ms[k] += ms;
  }
  cudaGetLastError();
  b->timing_pending = false;
}

// the I/O block for the members' present particle counts, allocated on
// first use and after a count change
memd_status batch_io_block(memd_batch* b) {
  const int64_t ntot = b->ioff.empty() ? 0 : b->ioff.back();
  if (b->io_ntot == ntot && b->io_host && b->io_dev) return MEMD_OK;
  free_io(b);
  const size_t bytes = (size_t)batch_io_bytes(ntot, (int)b->m.size());
  if (cudaHostAlloc((void**)&b->io_host, bytes, cudaHostAllocDefault) != cudaSuccess) {
    cudaGetLastError();
    b->io_host = nullptr;
    return bfail(b, MEMD_ERR_OOM, "page-locked batch I/O block");
  }
  std::memset(b->io_host, 0, bytes);
  if (b->alloc) {
    b->io_dev = b->alloc(b->alloc_user, bytes, (void*)b->stream);
  } else if (cudaMalloc(&b->io_dev, bytes) != cudaSuccess) {
    cudaGetLastError();
    b->io_dev = nullptr;
  }
  if (!b->io_dev) {
    cudaFreeHost(b->io_host);
    b->io_host = nullptr;
    return bfail(b, MEMD_ERR_OOM, "device batch I/O block");
  }
  b->io_ntot = ntot;
  return MEMD_OK;
}

// tables current for the members' present state (rebuilt when a member was
// re-initialised or stepped alone since they were built)
memd_status batch_refresh(memd_batch* b) {
  bool stale = false;
  for (size_t r = 0; r < b->m.size(); ++r) {
    memd_ctx* c = b->m[r];
    if (!c->initialised) return bfail(b, MEMD_ERR_STATE, "a member is not initialised");
    if (c->gen != b->gen[r] || c->cur != ((b->base[r] + b->bpar) & 1)) stale = true;
  }
  return stale ? build_tables(b) : MEMD_OK;
}

}  // namespace

// New members for an existing batch (the request server between rounds):
// the tables are rebuilt with the batch's field-kernel choice, stream-ordered
// behind the work already queued (the old tables and step graphs are released
// behind it too), with no stream or event created and no synchronisation.
// Members must share the batch's device, precision and stream.  Members that
// were not in the batch before get the per-particle constants of the
// batch's thermostat.
void memd_batch_set_overlap(memd_batch* b, bool overlap) {
  if (b->overlap == overlap) return;
  drop(b);  // the step graphs hold the launch order
  b->overlap = overlap;
}

memd_status memd_batch_update_members(memd_batch* b, int32_t count, memd_ctx* const* members) {
  if (!b || count < 1 || !members) return MEMD_ERR_INVALID;
  for (int r = 0; r < count; ++r) {
    const memd_ctx* c = members[r];
    if (!c || !c->initialised || c->device != b->device || c->prec != b->prec ||
        c->stream != b->stream)
      return bfail(b, MEMD_ERR_INVALID, "member does not fit the batch");
  }
  BCK(cudaSetDevice(b->device));
  harvest(b);
  std::vector<memd_ctx*> old = b->m;
  b->m.assign(members, members + count);
  b->gen.assign(count, -1);
  b->base.assign(count, 0);
  if (b->g_thermo >= 0)
    for (memd_ctx* c : b->m)
      if (std::find(old.begin(), old.end(), c) == old.end()) {
        launch_particle_constants(memd_step_params(c, b->g_thermo, b->g_gamma, b->g_kT), c->P,
                                  b->stream);
        c->sig_ready = false;
      }
  free_io(b);
  return build_tables(b, false);
}

// the batch, with its field tiles autotuned (tune) or the defaults
memd_status memd_batch_create_opt(int32_t count, memd_ctx* const* members, memd_batch** out,
                                  bool tune, int kind) {
  if (!out) return MEMD_ERR_INVALID;
  *out = nullptr;
  if (count < 1 || !members) return MEMD_ERR_INVALID;
  memd_batch* b = new memd_batch();
  for (int r = 0; r < count; ++r) {
    memd_ctx* c = members[r];
    if (!c || !c->initialised || c->device != members[0]->device ||
        c->prec != members[0]->prec || c->stream != members[0]->stream) {
      delete b;
      return MEMD_ERR_INVALID;
    }
    b->m.push_back(c);
  }
  b->gen.assign(count, -1);
  b->base.assign(count, 0);
  b->prec = members[0]->prec;
  b->device = members[0]->device;
  b->stream = members[0]->stream;
  b->alloc = members[0]->alloc;
  b->free_fn = members[0]->free_fn;
  b->alloc_user = members[0]->alloc_user;
  memd_status s = MEMD_OK;
  if (cudaSetDevice(b->device) != cudaSuccess ||
      cudaStreamCreateWithFlags(&b->side, cudaStreamNonBlocking) != cudaSuccess ||
      cudaEventCreateWithFlags(&b->fork, cudaEventDisableTiming) != cudaSuccess ||
      cudaEventCreateWithFlags(&b->join, cudaEventDisableTiming) != cudaSuccess ||
      cudaEventCreateWithFlags(&b->io_dep, cudaEventDisableTiming) != cudaSuccess ||
      cudaEventCreateWithFlags(&b->io_join, cudaEventDisableTiming) != cudaSuccess ||
      cudaEventCreate(&b->ev0) != cudaSuccess || cudaEventCreate(&b->ev1) != cudaSuccess ||
      [&] {
        for (auto& e : b->evp)
          if (cudaEventCreate(&e) != cudaSuccess) return true;
        return false;
      }()) {
    s = MEMD_ERR_CUDA;
  } else {
    // members' own queued work comes first
    for (memd_ctx* c : b->m) cudaStreamSynchronize(c->stream);
    b->f_pf = b->prec == MEMD_FP32 ? kBatchPF32 : kBatchPF64;
    b->f_kind = kind;
    if (kind == MEMD_FIELD_ROWS) b->f_rows = 256;
    // members that all fix the same row-kernel width (memd_options.field_shape)
    // fix the batch's: the row kernel with that width, untuned
    int fixed_rows = kind != MEMD_FIELD_SITE && b->m[0]->field_kernel == MEMD_FIELD_ROWS
                         ? b->m[0]->field_shape[3]
                         : 0;
    for (const memd_ctx* c : b->m)
      if (c->field_kernel != MEMD_FIELD_ROWS || c->field_shape[3] != fixed_rows) fixed_rows = 0;
    if (fixed_rows) {
      b->f_kind = MEMD_FIELD_ROWS;
      b->f_rows = fixed_rows;
      s = build_tables(b);
    } else {
      s = tune ? autotune_batch(b) : build_tables(b);
    }
  }
  if (s != MEMD_OK) {
    memd_batch_destroy(b);
    return s;
  }
  *out = b;
  return MEMD_OK;
}

extern "C" {

void memd_batch_destroy(memd_batch* b) {
  if (!b) return;
  cudaSetDevice(b->device);
  if (b->stream) cudaStreamSynchronize(b->stream);
  drop(b);
  free_tables(b);
  free_io(b);
  if (b->fork) cudaEventDestroy(b->fork);
  if (b->join) cudaEventDestroy(b->join);
  if (b->io_dep) cudaEventDestroy(b->io_dep);
  if (b->io_join) cudaEventDestroy(b->io_join);
  if (b->ev0) cudaEventDestroy(b->ev0);
  if (b->ev1) cudaEventDestroy(b->ev1);
  for (auto& e : b->evp)
    if (e) cudaEventDestroy(e);
  if (b->side) cudaStreamDestroy(b->side);
  delete b;
}

memd_status memd_batch_create(int32_t count, memd_ctx* const* members, memd_batch** out) {
  return memd_batch_create_opt(count, members, out, true, MEMD_FIELD_AUTO);
}

memd_status memd_batch_create_kernel(int32_t count, memd_ctx* const* members,
                                     int32_t field_kernel, memd_batch** out) {
  if (field_kernel != MEMD_FIELD_AUTO && field_kernel != MEMD_FIELD_SITE &&
      field_kernel != MEMD_FIELD_ROWS)
    return MEMD_ERR_INVALID;
  return memd_batch_create_opt(count, members, out, true, field_kernel);
}

memd_status memd_batch_step(memd_batch* b, int64_t nsteps, const memd_thermostat* th) {
  memd::NvtxRange nvtx_("memd_batch_step");
  if (!b) return MEMD_ERR_INVALID;
  if (nsteps < 0) return bfail(b, MEMD_ERR_INVALID, "negative step count");
  BCK(cudaSetDevice(b->device));
  // members re-initialised or stepped on their own since the tables were built
  {
    const memd_status s = batch_refresh(b);
    if (s != MEMD_OK) return s;
  }
  const int thermo = th ? 1 : 0;
  const double gamma = th ? th->gamma : 0.0, kT = th ? th->kT : 0.0;
  set_thermostat(b, thermo, gamma, kT);
  const bool timed = batch_timed(b);
  for (int64_t s = 0; s < nsteps; ++s) {
    const int par = b->bpar;
    harvest(b);
    if (b->single && !b->single_graph_ok) {
      // the cooperative launch could not be captured here: launched directly
      const memd_status r = record(b, par, thermo, gamma, kT, timed);
      if (r != MEMD_OK) return r;
      b->timing_pending = timed;
      b->bpar ^= 1;
      continue;
    }
    cudaGraphExec_t& gx = b->graph[par];
    if (!gx) {
      cudaGraph_t g = nullptr;
      BCK(cudaStreamBeginCapture(b->stream, cudaStreamCaptureModeThreadLocal));
      memd_status r = record(b, par, thermo, gamma, kT, timed);
      cudaError_t e = cudaStreamEndCapture(b->stream, &g);
      if (r != MEMD_OK) {
        if (g) cudaGraphDestroy(g);
        return r;
      }
      cudaError_t ie = e == cudaSuccess ? cudaGraphInstantiate(&gx, g, 0) : e;
      if (g) cudaGraphDestroy(g);
      if (ie != cudaSuccess) {
        gx = nullptr;
        if (!b->single) return bfail(b, MEMD_ERR_CUDA, "graph capture");
        cudaGetLastError();
        b->single_graph_ok = false;
        --s;  // this step again, launched directly
        continue;
      }
    }
    BCK(cudaGraphLaunch(gx, b->stream));
    b->timing_pending = timed;
    b->bpar ^= 1;
  }
  for (size_t r = 0; r < b->m.size(); ++r) b->m[r]->cur = (b->base[r] + b->bpar) & 1;
  return MEMD_OK;
}

memd_status memd_batch_synchronize(memd_batch* b) {
  if (!b) return MEMD_ERR_INVALID;
  BCK(cudaSetDevice(b->device));
  harvest(b);
  BCK(cudaStreamSynchronize(b->stream));
  if (b->single && b->d_sched) {
    // a wait of the single-launch step that ran out leaves its counts out of
    // step: start them afresh (the step is void)
    unsigned int err = 0;
    BCK(cudaMemcpy(&err, &b->d_sched->err, sizeof(err), cudaMemcpyDeviceToHost));
    if (err) {
      BCK(cudaMemset(b->d_sched, 0, sizeof(BatchSched)));
      BCK(cudaMemset(b->d_sync, 0, sizeof(RepSync) * b->m.size()));
      return bfail(b, MEMD_ERR_TIMEOUT, "a wait of the single-launch batch step ran out");
    }
  }
  for (memd_ctx* c : b->m) {
    const memd_status s = memd_check_err(c);
    if (s != MEMD_OK) return bfail(b, s, c->last_error);
  }
  return MEMD_OK;
}

memd_status memd_batch_set_timing(memd_batch* b, int32_t on) {
  if (!b) return MEMD_ERR_INVALID;
  BCK(cudaSetDevice(b->device));
  harvest(b);
  const int t = on ? 1 : 0;
  if (t != b->timing) {
    BCK(cudaStreamSynchronize(b->stream));
    drop(b);  // the step graphs hold (or lack) the timing events
    b->timing = t;
  }
  return MEMD_OK;
}

memd_status memd_batch_io_buffers(memd_batch* b, memd_batch_io* io) {
  if (!b || !io) return MEMD_ERR_INVALID;
  BCK(cudaSetDevice(b->device));
  memd_status s = batch_refresh(b);
  if (s == MEMD_OK) s = batch_io_block(b);
  if (s != MEMD_OK) return s;
  const IoLayout L = io_layout(b->io_ntot);
  io->pos = (double*)(b->io_host + L.pos);
  io->vel = (double*)(b->io_host + L.vel);
  io->img = (int32_t*)(b->io_host + L.img);
  io->f = (double*)(b->io_host + L.f);
  io->offsets = b->ioff.data();
  io->n_total = b->io_ntot;
  return MEMD_OK;
}

memd_status memd_batch_step_io(memd_batch* b, int32_t load, int64_t nsteps,
                               const memd_thermostat* th) {
  memd::NvtxRange nvtx_("memd_batch_step_io");
  if (!b) return MEMD_ERR_INVALID;
  if (nsteps < 0) return bfail(b, MEMD_ERR_INVALID, "negative step count");
  BCK(cudaSetDevice(b->device));
  memd_status s = batch_refresh(b);
  if (s == MEMD_OK) s = batch_io_block(b);
  if (s != MEMD_OK) return s;
  const int R = (int)b->m.size();
  const int64_t ntot = b->io_ntot;
  const IoLayout L = io_layout(ntot);
  const cudaStream_t st = b->stream;
  auto member_errors = [&]() -> memd_status {
    const unsigned int* err = (const unsigned int*)(b->io_host + L.err);
    for (int r = 0; r < R; ++r)
      if (err[r]) {
        const memd_status e = memd_check_err(b->m[r]);
        if (e != MEMD_OK) return bfail(b, e, b->m[r]->last_error);
      }
    return MEMD_OK;
  };
  if (load && nsteps == 1 && ntot > 0 && !b->single && b->overlap && !batch_timed(b)) {
    // the usual host loop: one graph a call, the copies beside the step
    const int thermo = th ? 1 : 0;
    const double gamma = th ? th->gamma : 0.0, kT = th ? th->kT : 0.0;
    set_thermostat(b, thermo, gamma, kT);
    harvest(b);
    const int par = b->bpar;
    cudaGraphExec_t& gx = b->io_graph[par];
    if (!gx) {
      cudaGraph_t g = nullptr;
      BCK(cudaStreamBeginCapture(st, cudaStreamCaptureModeThreadLocal));
      const memd_status r = record_io(b, par, thermo, gamma, kT);
      const cudaError_t e = cudaStreamEndCapture(st, &g);
      if (r != MEMD_OK) {
        if (g) cudaGraphDestroy(g);
        return r;
      }
      const cudaError_t ie = e == cudaSuccess ? cudaGraphInstantiate(&gx, g, 0) : e;
      if (g) cudaGraphDestroy(g);
      if (ie != cudaSuccess) {
        gx = nullptr;
        return bfail(b, MEMD_ERR_CUDA, "I/O step graph capture");
      }
    }
    BCK(cudaGraphLaunch(gx, st));
    b->bpar ^= 1;
    for (size_t r = 0; r < b->m.size(); ++r) b->m[r]->cur = (b->base[r] + b->bpar) & 1;
    BCK(cudaStreamSynchronize(st));
    return member_errors();
  }
  if (load && ntot > 0) {
    // positions, velocities and image counters of every member: one copy
    BCK(cudaMemcpyAsync(b->io_dev, b->io_host, (size_t)L.f, cudaMemcpyHostToDevice, st));
    launch_io_unpack_batch(b->d_desc, b->d_ioff, R, ntot, b->io_dev, st);
    BCK(cudaGetLastError());
  }
  s = memd_batch_step(b, nsteps, th);
  if (s != MEMD_OK) return s;
  launch_io_pack_batch(b->d_desc, b->d_ioff, R, ntot, b->io_dev, st);
  BCK(cudaGetLastError());
  BCK(cudaMemcpyAsync(b->io_host, b->io_dev, (size_t)batch_io_bytes(ntot, R),
                      cudaMemcpyDeviceToHost, st));
  BCK(cudaStreamSynchronize(st));
  return member_errors();
}

memd_status memd_batch_set_engine(memd_batch* b, int32_t engine, int32_t field_ctas,
                                  int32_t item_planes) {
  if (!b) return MEMD_ERR_INVALID;
  if (engine < MEMD_STEP_AUTO || engine > MEMD_STEP_SINGLE || item_planes < 0)
    return bfail(b, MEMD_ERR_INVALID, "bad engine options");
  BCK(cudaSetDevice(b->device));
  harvest(b);
  BCK(cudaStreamSynchronize(b->stream));
  b->engine = engine;
  b->bs_field_ctas = field_ctas;
  b->bs_item_planes = item_planes;
  const memd_status s = build_tables(b);
  if (s != MEMD_OK) return s;
  if (engine == MEMD_STEP_SINGLE && !b->single)
    return bfail(b, MEMD_ERR_INVALID, "the single-launch step cannot run this batch");
  return MEMD_OK;
}

memd_status memd_batch_kernel_stats(memd_batch* b, memd_kernel_stats* out) {
  if (!b || !out) return MEMD_ERR_INVALID;
  harvest(b);
  std::memset(out, 0, sizeof(*out));
  out->field_ms = b->field_ms;
  out->field_launches = b->field_launches;
  out->field_bytes = b->field_bytes;
  out->launches_per_step = b->single ? 1 : 4;
  out->step_single = b->single ? 1 : 0;
  out->field_tma = 0;
  out->field_ty = b->f_ty;
  out->field_tma = 0;
  out->field_tx = b->f_w;
  out->field_zchunk = b->f_z;
  out->field_site = b->f_rows > 0 ? 0 : b->f_pf;
  out->field_rows = b->f_rows;
  for (int k = 0; k < 3; ++k) {
    out->phase_ms[k] = b->phase_ms[k];
    b->phase_ms[k] = 0.0;
  }
  b->field_ms = 0.0;
  b->field_launches = 0;
  return MEMD_OK;
}

}  // extern "C"
