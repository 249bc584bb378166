// memd_ctx.cuh -- the context behind the opaque memd_ctx handle, shared by
// the single-system API (memd_api.cu) and the batched replicas
// (memd_batch.cu).  Host-side only.
#pragma once

#include <string>
#include <utility>
#include <vector>

#include "memd.h"
#include "memd_internal.cuh"

struct memd_ctx {
  using FusedCfg = memd::FusedCfg;
  using TmaMaps = memd::TmaMaps;
  using Mesh = memd::Mesh;
  using DevState = memd::DevState;
  using Particles = memd::Particles;
  Mesh mesh;
  double Vbox = 0, c = 0, dt = 0;
  int prec = 0, self_mode = 1, dipole_corr = 1, relax_maxit = 200000, use_graphs = 1;
  int time_kernels = 0;
  double relax_tol = 1e-12;
  unsigned long long seed = 0;
  int device = 0;
  cudaStream_t stream = nullptr;
  bool own_stream = false;
  memd_alloc_fn alloc = nullptr;
  memd_free_fn free_fn = nullptr;
  void* alloc_user = nullptr;
  std::vector<std::pair<void*, size_t>> blocks;
  std::string last_error;
  // field arrays: D and B double-buffered for the fused update; cur is the
  // buffer that holds the present state
  void* Dbuf[2] = {nullptr, nullptr};
  void* Bbuf[2] = {nullptr, nullptr};
  int cur = 0;
  void* ie = nullptr;
  double* ie64 = nullptr;
  long long* Lg = nullptr;
  long long* Tb = nullptr;
  DevState* ds = nullptr;
  double* red = nullptr;  // reduction partials (4 x reduce_blocks) + 32 scalars
  double G[8] = {0};
  double Minv[9] = {0};
  double eps_eff_inv[9] = {0};  // exact inverse of the effective permittivity (Minv symmetrised)
  double* psi = nullptr;        // cell-problem potentials of the scalar solver (3V), or null
  double* pin = nullptr;        // memd_set_particles staging (3n doubles + 3n ints)
  long long* Tb2 = nullptr;     // second transfer buffer of the single-launch step
  bool pending = false;         // transfers of the last single-launch step not yet applied
  // particles
  Particles P{};
  bool initialised = false;
  bool eps_ready = false;
  unsigned int* err_host = nullptr;  // page-locked copy of the error word (memd_step_host)
  // the host I/O block of memd_step_io: page-locked on the host, mirrored on
  // the device; sized for io_n particles
  unsigned char* io_host = nullptr;
  void* io_dev = nullptr;
  int64_t io_n = -1;
  // the row kernel's tables for this context alone (built when tuned)
  memd::RepDesc* rows_desc = nullptr;
  memd::RowSeg* rows_segs = nullptr;
  int* rows_first = nullptr;
  int rows_nctas = 0;
  int rows_nt = 0;       // a permittivity is mapped (memd_set_eps restores it on failure)
  // step graphs, one per buffer parity
  cudaGraphExec_t graph[2] = {nullptr, nullptr};
  // memd_step_io's whole round trip (copy in, unpack, step, pack, copy out)
  // as one graph per buffer parity; io_graph_ok false once capture failed
  cudaGraphExec_t io_graph[2] = {nullptr, nullptr};
  bool io_graph_ok = true;
  int step_engine = 0;   // MEMD_STEP_*
  int apply_mode = 0;    // MEMD_APPLY_*
  int coop_grid = 0;     // CTAs of the single-launch step (0: unsupported)
  bool coop = false;     // the steps run as one cooperative launch
  bool coop_graph_ok = true;  // its launch can be captured in a graph
  int graph_thermo = -1;
  double graph_gamma = 0, graph_kT = 0;
  cudaStream_t side = nullptr;
  cudaEvent_t fork = nullptr, join = nullptr;
  cudaEvent_t ev0 = nullptr, ev1 = nullptr;
  bool timing_pending = false;
  double field_ms = 0;
  long long field_launches = 0;
  int relax_iters_last = 0;
  int gen = 0;  // bumped by every memd_init_field (batches rebuild their tables)
  FusedCfg fcfg{8, 1, 0, 0, 0};
  bool fcfg_ready = false;  // fcfg autotuned (at the first step that needs it)
  int field_kernel = 0;
  int field_shape[4] = {0, 0, 0, 0};  // {ty, zchunk, planes_ahead, rows_nt}; 0: autotuned
  unsigned long long wait_ns = memd::kBarrierWaitNs;  // grid-barrier wait bound (memd_inject)
  TmaMaps tma{};
  bool tma_ok = false;
  bool sig_ready = false;
  void* D() const { return Dbuf[cur]; }
  void* B() const { return Bbuf[cur]; }
};


// helpers of memd_api.cu used by memd_batch.cu
void* memd_dalloc(memd_ctx* c, size_t bytes);
void memd_dfree(memd_ctx* c, void* p);
size_t memd_esz(const memd_ctx* c);
memd::StepParams memd_step_params(const memd_ctx* c, int thermo, double gamma, double kT);
memd_status memd_check_err(memd_ctx* c);
memd_status memd_flush(memd_ctx* c);  // apply pending transfers of the single-launch step
// memd_mg.cu: effective permittivity and initial field through the scalar
// potential (multigrid-preconditioned CG on the vertices)
namespace memd {
memd_status mg_eps_eff(memd_ctx* c, double* psi, double eps_eff[9], double tol, int maxit);
// on the calling thread from now on: the cell problems of mg_eps_eff solved
// in turn (one solver) instead of at once (three solvers, streams, threads)
void memd_mg_cells_in_turn(bool on);
memd_status mg_relax(memd_ctx* c, double* D64, const double* psi, const double eps_eff_inv[9],
                     double tol, int maxit, int* iters);
// memd_rows.cu: the row kernel's work split for a set of contexts (false
// when one of them does not fit the kernel)
bool rows_plan(const std::vector<memd_ctx*>& m, int prec, int nt, int nctas,
               std::vector<RowSeg>& segs, std::vector<int>& first);
}  // namespace memd
// memd_batch.cu, for the server: a batch whose field kernel is autotuned
// (tune) or left at its defaults, within the family `kind` (MEMD_FIELD_AUTO,
// MEMD_FIELD_SITE or MEMD_FIELD_ROWS)
memd_status memd_batch_create_opt(int32_t count, memd_ctx* const* members, memd_batch** out,
                                  bool tune, int kind);
// new members for a batch, its tables rebuilt behind the queued work (no
// synchronisation); members share the batch's device, precision and stream
memd_status memd_batch_update_members(memd_batch* b, int32_t count, memd_ctx* const* members);
// whether the deposition runs beside the field pass (the default) or after
// it on the batch's stream; the step graphs are rebuilt at the next step
void memd_batch_set_overlap(memd_batch* b, bool overlap);
