// memd_internal.cuh -- shared declarations of the MEMD CUDA library (sm_103a).
//
// Lattice conventions (Sec. II, Fig. 2): vertex v = (i, j, k) at flat index
// i + nx (j + ny k); link (d, v) joins v to v + e_d and is stored at d V + v;
// plaquette (d, v) has normal e_d, spans e_{d+1}, e_{d+2} from v and is stored
// at d V + v.  Fixed point: S = 2^16 sub-cell steps; charge and flux unit
// e 2^-48.
#pragma once

#include <cuda.h>
#include <cuda_runtime.h>
#include <nvtx3/nvToolsExt.h>
#include <stdint.h>

namespace memd {

// NVTX range around a host-side phase (create, init, step, batch step,
// server round, request setup, autotuning): visible in a profiler's
// timeline, a no-op without one
struct NvtxRange {
  explicit NvtxRange(const char* name) { nvtxRangePushA(name); }
  ~NvtxRange() { nvtxRangePop(); }
  NvtxRange(const NvtxRange&) = delete;
  NvtxRange& operator=(const NvtxRange&) = delete;
};

constexpr int kWBits = 16;
constexpr int64_t kS = int64_t(1) << kWBits;

struct Mesh {
  int n[3];
  int64_t V;
  double a;
  double L[3];
  double inv_a;  // 1 / a; used instead of the division when a is a power of two
  int a_pow2;    // (x * inv_a == x / a exactly then)
  double inv_aS; // S / a (exact when a is a power of two)
};

// The transfer buffer and the ledger of a system share one allocation of
// 6 V int64 words, vertex major: the links (0, v), (1, v), (2, v) leaving
// vertex v are pairs 3 v, 3 v + 1, 3 v + 2, and pair k holds the transfer
// word at [kLT k] and the ledger word at [kLT k + 1].  The transfer
// application reads one and adds into the other, which then share a sector;
// a charge's links (the twelve edges of its cell) sit at seven vertices in
// four rows, a few L2 lines, where the fields' component-major order would
// spread them over a dozen.  Kernels index both arrays with this stride
// (the ledger pointer is the allocation plus one word).
constexpr int kLT = 2;
// pair of link (d, v)
__host__ __device__ inline int64_t tl_pair(int d, int64_t v) { return 3 * v + d; }
// pair of the link with field index l = d V + v
__host__ __device__ inline int64_t tl_pair_of(int64_t l, int64_t V) {
  const int d = l >= 2 * V ? 2 : (l >= V ? 1 : 0);
  return tl_pair(d, l - d * V);
}
// The word of link (d, v) in a transfer buffer: the transfer word of its
// pair (cmV == 0), or, in the single-launch step's own buffers of transfer
// words only (cmV == V), component major at d V + v, where the field tiles'
// dense reads of a plane's pending transfers are coalesced.
__host__ __device__ inline int64_t tw_index(int d, int64_t v, int64_t cmV) {
  return cmV ? d * cmV + v : kLT * tl_pair(d, v);
}

// error bits raised by kernels into a device word
enum : unsigned int {
  kErrCellJump = 1u,
  kErrGauss = 2u,
  kErrOverflow = 4u,
  kErrNonFinite = 8u,
  kErrTimeout = 16u,
};

// Small device-resident state shared by the step kernels.
struct DevState {
  unsigned long long Pacc[3];  // sum q U (int64 bits) of the current positions
  long long Plast[3];          // P of the last completed update
  long long step;              // steps since init (Langevin counter)
  unsigned int err;            // kErr* bits
  unsigned int ticket;         // blocks of the gather that have finished
  unsigned long long bar_arrivals;  // grid barrier of the single-launch step: CTA arrivals
                                    // since init (grows by the grid size a barrier)
  long long lsum[3];           // scratch: sum of the ledger per component
  double scal[16];             // scratch scalars for the relaxation
};

__host__ __device__ inline int64_t vindex(const Mesh& m, int i, int j, int k) {
  return (int64_t)i + (int64_t)m.n[0] * ((int64_t)j + (int64_t)m.n[1] * k);
}

__host__ __device__ inline int wrapi(int i, int n) {
  i %= n;
  return i < 0 ? i + n : i;
}

// ------------------------------------------------------------ L2 priorities
// Cache-priority policies (PTX createpolicy, sm_80 and later).  The transfer
// and ledger words, scattered by the particle kernels' atomics and touched
// again by the next particle kernel of the step, are kept in L2 (evict_last);
// the field planes that the stencil streams through once a step leave first
// (evict_first).  These are hints: no value and no order of operations
// changes.  The asm is not volatile, so one policy per thread is hoisted.
__device__ __forceinline__ unsigned long long l2_policy_last() {
  unsigned long long p;
  asm("createpolicy.fractional.L2::evict_last.b64 %0, 1.0;" : "=l"(p));
  return p;
}
__device__ __forceinline__ unsigned long long l2_policy_first() {
  unsigned long long p;
  asm("createpolicy.fractional.L2::evict_first.b64 %0, 1.0;" : "=l"(p));
  return p;
}
// atomicAdd without a result (relaxed, device scope) under an L2 policy
__device__ __forceinline__ void red_add_hint(unsigned long long* a, unsigned long long v,
                                             unsigned long long pol) {
  asm volatile("red.global.add.L2::cache_hint.u64 [%0], %1, %2;" ::"l"(a), "l"(v), "l"(pol)
               : "memory");
}
// atomicExch (relaxed, device scope) under an L2 policy
__device__ __forceinline__ unsigned long long exch_hint(unsigned long long* a, unsigned long long v,
                                                        unsigned long long pol) {
  unsigned long long r;
  asm volatile("atom.global.exch.L2::cache_hint.b64 %0, [%1], %2, %3;"
               : "=l"(r)
               : "l"(a), "l"(v), "l"(pol)
               : "memory");
  return r;
}

// ------------------------------------------------------------ field kernels
// (memd_field.cu)
void launch_curl_B(const Mesh& m, int prec, void* B, const void* D, const void* ie,
                   double coef, cudaStream_t st);
void launch_curl_D(const Mesh& m, int prec, void* D, const void* B, double coef,
                   cudaStream_t st);
// fused B then D update with double-buffered fields: tile height ty (4, 8
// or 16 rows of 32) and z planes per CTA; zchunk <= 0 takes the default
struct FusedCfg {
  int ty;
  int zchunk;
  int tma;   // 1: TMA-staged kernel (memd_tma.cu)
  int site;  // k >= 1: one-thread-per-site kernel (k_fused_site), loads k planes ahead;
             // 0: k_fused_curl
  int rows;  // nt > 0: the row kernel (memd_rows.cu) with nt threads a CTA
};
void launch_fused_curl(const Mesh& m, int prec, const void* Din, const void* Bin, const void* ie,
                       void* Dout, void* Bout, double cB, double cD, FusedCfg cfg,
                       cudaStream_t st);
FusedCfg fused_default(const Mesh& m);
// candidate shapes for the autotuner; returns how many were written
int fused_candidates(const Mesh& m, int prec, FusedCfg* out, int cap);
// TMA-staged fused update (memd_tma.cu): usable when x rows are 16-byte
// multiples; one 4-D tensor map per array, buffer parity and tile height
struct TmaMaps {
  CUtensorMap D[2][3], B[2][3], ie[3];
  static int index(int ty) { return ty == 4 ? 0 : (ty == 16 ? 2 : 1); }
  static int ty(int t) { return t == 0 ? 4 : (t == 2 ? 16 : 8); }
};
bool tma_supported(const Mesh& m, int prec);
bool tma_make_maps(const Mesh& m, int prec, void* const D[2], void* const B[2], void* ie,
                   TmaMaps* out);
void launch_fused_tma(const Mesh& m, int prec, const TmaMaps& maps, int par, const void* Din,
                      const void* Bin, const void* ie, void* Dout, void* Bout, double cB,
                      double cD, FusedCfg cfg, unsigned int* err, cudaStream_t st);
// FP64 helpers of the relaxation: w = sign * circulation(ie * u) per plaquette
void launch_circ64(const Mesh& m, double* w, const double* u, const double* ie,
                   double sign, cudaStream_t st);
// u = transpose of the circulation map applied to a plaquette field p
void launch_curlT64(const Mesh& m, double* u, const double* p, cudaStream_t st);
// fused PCG iteration (memd_field.cu): w = circ(ie u) with CTA shares of p.w;
// the update with shares of r.z and max|r|; the new direction.  Scalar slots
// of sc: 14 frozen flag, 15 tolerance, 4 max|E|; part_* hold reduce_blocks()
// CTA shares each.
void launch_cg_apply(const Mesh& m, double* w, const double* u, const double* ie,
                     const double* p, double* part, cudaStream_t st);
void launch_cg_update(int64_t n, double* D, const double* u, double* r, const double* w,
                      double* z, const double* diag, const double* part_pw, const double* sc,
                      int rz_slot, double* part_rz, double* part_rmax, cudaStream_t st);
void launch_cg_direction(int64_t n, double* p, const double* z, double* sc, const double* part_rz,
                         const double* part_rmax, int rz_new, int rz_old, cudaStream_t st);
// diag_p = sum of ie over the 4 links of each plaquette
void launch_plaquette_diag(const Mesh& m, double* diag, const double* ie, cudaStream_t st);

// --------------------------------------------------- setup / init kernels
// (memd_setup.cu)
struct EpsDesc {
  int kind;
  int axis;
  double p[8];
};
void launch_eps_links(const Mesh& m, const EpsDesc& e, const double* values, double* ie64,
                      unsigned int* err, cudaStream_t st);
void launch_cast(int prec, void* dst, const double* src, int64_t count, cudaStream_t st);
void launch_widen(int prec, double* dst, const void* src, int64_t count, cudaStream_t st);
// Green's table: 8 values into G (device), using `partial` scratch of
// green_partials() doubles
int green_partials();
void launch_green(const Mesh& m, double* partial, double* G, cudaStream_t st);
// Gauss scan of vertex charges Q into the ledger (Fig. 1); scratch of
// scan_scratch(m) int64
int64_t scan_scratch(const Mesh& m);
void launch_gauss_scan(const Mesh& m, const long long* Q, long long* Lg, long long* scratch,
                       unsigned int* err, cudaStream_t st);
// D64 = Lg scale + shift_d with shift_d = -P_d / Vbox - mean(Lg_d) scale
void launch_init_D(const Mesh& m, double* D64, const long long* Lg, DevState* ds,
                   double scale, double Vbox, cudaStream_t st);
void launch_ledger_sums(const Mesh& m, const long long* Lg, DevState* ds, cudaStream_t st);
// permittivity from the salt density: rho = |q| density (from its
// fixed-point deposit Q), smoothed along x, y, z by the weights w[0..2R]
// (sigma > 0), its sum into sum[0] (partials in part), then eps per vertex
// from rule {eps0, slope, lo, hi}; tmp is V doubles of scratch
void launch_salt_eps(const Mesh& m, const long long* Q, double* rho, double* tmp,
                     const double* w, int R, double sigma, double* part, double* sum,
                     const double rule[4], double* eps, cudaStream_t st);
// zero the transfer words of a transfer buffer of count links (stride kLT)
void launch_clear_transfers(long long* T, int64_t count, cudaStream_t st);

// deterministic FP64 reductions (memd_setup.cu)
int reduce_blocks();
// partial[b] = block sums of x[i] * y[i] (y may be NULL: sum of x)
void launch_dot(const double* x, const double* y, int64_t n, double* partial, cudaStream_t st);
// partial[b] = block max of |x[i]| (|x[i] y[i]| when y is given)
void launch_absmax(const double* x, const double* y, int64_t n, double* partial,
                   cudaStream_t st);
// out[0] = op over partial[0..reduce_blocks())  (op 0 = sum, 1 = max)
void launch_finish(const double* partial, int op, double* out, cudaStream_t st);

// ------------------------------------------------------- particle kernels
// (memd_particles.cu, built with -fmad=false)
struct Particles {
  int64_t n;
  double* x;
  double* v;
  double* m;
  double* F;
  double* Ft;
  int* img;
  int* q;
  int* mv;      // kMoveInts ints per particle: old cell (3), new cell (3) and new
                // sub-cell step (3) of the last move
  double* h;    // dt / (2 m): half-kick factor
  double* sig;  // sqrt(2 gamma m kT / dt): Langevin noise amplitude
  double* gm;   // -gamma m: Langevin friction per unit velocity
};
constexpr int kMoveInts = 9;
struct StepParams {
  double dt;
  double coefB;   // dt / a
  double coefD;   // c^2 dt / a
  double scale;   // 2^-48 / a^2
  double Vbox;
  double inv_V;     // 1 / Vbox
  double self_pre;  // 1 / (2 a^2): self-energy force q^2 ie sum / (2 a a)
  double dip_unit;  // a / S: length of one sub-cell step
  double G[8];
  double Minv[9];
  double Mdip[9];   // Minv (a / S) / Vbox: dipole force per unit charge per fixed-point P
  // the same constants rounded to FP32, for the force terms with FP32 fields
  // (the values a conversion at each use would give)
  float Gf[8];
  float Mdipf[9];
  float self_pref;
  int self_mode;
  int dipole_corr;
  int thermo;
  double gamma;
  double kT;
  unsigned long long seed;
  unsigned long long wait_ns;  // bound of the single-launch step's grid-barrier wait
};
constexpr unsigned long long kBarrierWaitNs = 200000000ull;  // 0.2 s
// single-launch step (memd_particles.cu): the whole time step in one
// cooperative launch, for systems small enough that launch gaps dominate
constexpr int kCoopFieldWarps = 11;                  // 34 x 10 site tile of 8 rows
constexpr int kCoopThreads = 32 * (kCoopFieldWarps + 1);
int coop_grid(int prec, int device);                 // CTAs of one cooperative launch, 0 if none
int coop_zchunk(const Mesh& m, int grid);
cudaError_t launch_step_coop(const Mesh& m, int prec, const StepParams& sp, Particles p,
                             const void* Din, const void* Bin, const void* ie, void* Dout,
                             void* Bout, const double* ie64, long long* Tprev, long long* Tcur,
                             long long* Lg, DevState* ds, int grid, int zchunk, cudaStream_t st);
void launch_fold_init(const Mesh& m, Particles p, const double* pos_in, const int* img_in,
                      unsigned int* err, cudaStream_t st);
// byte offsets of the host I/O block of n particles (memd_step_io)
// The host I/O block of n particles: positions, image counters and
// velocities (a step's inputs: the range [0, f)), then forces and the error
// word(s).  Positions and image counters are final once the drift is done
// and form the range [0, vel), which can go back while the step's gather
// runs; velocities, forces and errors, the range [vel, end), after it.
struct IoLayout {
  int64_t pos, vel, img, f, err, bytes;
};
__host__ __device__ inline IoLayout io_layout(int64_t n) {
  IoLayout L;
  L.pos = 0;
  L.img = 24 * n;
  L.vel = L.img + ((12 * n + 7) / 8) * 8;
  L.f = L.vel + 24 * n;
  L.err = L.f + 24 * n;
  L.bytes = L.err + 8;
  return L;
}
// what a pack writes: everything, the moved part (positions, image
// counters) or the rest (velocities, forces, error words)
enum : int { kIoAll = 0, kIoMoved = 1, kIoRest = 2 };
void launch_io_unpack(const Mesh& m, Particles p, const void* io, unsigned int* err,
                      cudaStream_t st);
void launch_io_pack(Particles p, void* io, const unsigned int* err, cudaStream_t st);
void launch_cic(const Mesh& m, Particles p, long long* Q, long long bg, cudaStream_t st);
// cloud-in-cell deposit of |q| (int64, e 2^-48) at the vertices
void launch_cic_abs(const Mesh& m, Particles p, long long* Q, cudaStream_t st);
void launch_dipole(const Mesh& m, Particles p, DevState* ds, cudaStream_t st);
void launch_kick_drift_deposit(const Mesh& m, const StepParams& sp, Particles p,
                               long long* Tb, DevState* ds, cudaStream_t st);
void launch_move_deposit(const Mesh& m, Particles p, const double* pos_new,
                         const int* img_new, long long* Tb, DevState* ds, cudaStream_t st);
// cmV: the layout of Tb (tw_index); the ledger Lg is always the pairs'
void launch_apply(const Mesh& m, int prec, Particles p, long long* Tb, long long* Lg, void* D,
                  double scale, cudaStream_t st, int64_t cmV = 0);
// the same over every one of nlinks transfer words (one pass, no particle
// data); identical results.  Cheaper when the mesh has few links per charge.
void launch_apply_dense(int prec, int64_t nlinks, long long* Tb, long long* Lg, void* D,
                        double scale, cudaStream_t st);
// MEMD_APPLY_AUTO is the sparse pass.  A dense pass reads 24 B a vertex and
// rewrites the words that carry a transfer; the sparse pass costs ~0.25-0.3 ns
// a charge on GB300 (12 atomic round trips per quad, issued together).
// Measured a step: the 64^3 system with 32768 charges 44.1 us dense vs 44.8
// sparse (within run-to-run spread); 64 replicas with 124k charges and
// fields larger than L2, 161.5 vs 142.0 (the 71 MB of transfer words cost
// more than the exchanges).
inline bool apply_dense(int mode) { return mode == 2; }  // MEMD_APPLY_DENSE
// finish: 0 nothing, 1 close the update (P of this state, clear the
// accumulator), 2 also advance the step counter; done by the last CTA
void launch_gather(const Mesh& m, int prec, const StepParams& sp, Particles p, const void* D,
                   const void* ie, const double* ie64, DevState* ds, int kick, int finish,
                   cudaStream_t st);
void launch_step_end(DevState* ds, int advance, cudaStream_t st);

// ------------------------------------------------------- batched replicas
// One independent system of a batch, as the batched kernels see it.
struct RepDesc {
  Mesh m;
  StepParams sp;
  Particles P;
  void* D[2];
  void* B[2];
  void* ie;
  double* ie64;
  long long* Lg;
  long long* Tb;
  DevState* ds;
  int f_first, f_tx, f_ty, f_zchunk;  // field tiles: first CTA, tiles along x, y; planes per CTA
  int p_first, p_ctas;                // particle CTAs of the quad kernels
  int pw_first, pw_ctas;              // and of the one-thread-per-charge kernels
  int b_nf, b_np, b_nc;               // single-launch step: field items, particle items,
                                      // particle chunks (kBatchStepThreads quad lanes)
};
constexpr int kBatchTY = 8;            // default tile height of the batched field kernel
constexpr int kBatchPF32 = 2;          // its prefetch depth in planes, FP32 fields
constexpr int kBatchPF64 = 1;          // and FP64 fields (register bound)
constexpr int kBatchZ = 8;             // and its planes per CTA
constexpr int kBatchQuadThreads = 128;  // 32 particles per CTA in the batched quad kernels
// Deposition and gather run one thread per charge (kWideThreads a CTA) from
// kWideMinCharges charges a system (a batch: charges over all members) on:
// there the instruction count per charge, not latency, bounds them; below
// it four lanes per charge split each charge's serial FP64 chain.
constexpr int kWideThreads = 128;
constexpr int64_t kWideMinCharges = 16384;
// One segment of the row kernel's work (memd_rows.cu): rows y0 .. y0 + rows - 1
// of replica rep, planes za .. zb - 1.
struct RowSeg {
  int rep, y0, rows, za, zb;
};
// row kernel: sites a thread (16 bytes of the field type), CTAs an SM, launch
size_t rows_smem_bytes(int nt, size_t esz);
int rows_sites_per_thread(int prec);
int rows_occupancy(int prec, int nt);
cudaError_t launch_rows_batch(int prec, const RepDesc* desc, const RowSeg* segs,
                              const int* seg_first, int nctas, int nt, int par, cudaStream_t st);
// ------------------------------------------- single-launch batch step
// (memd_particles.cu) The whole step of every replica in one cooperative
// launch of persistent CTAs that claim work: field segments (a row tile over
// a range of planes) and deposition items from two device queues, transfer
// application and gather items of a replica from that replica's own claim
// counts, once ready.  A particle item is kBatchChunksPerItem chunks of
// kBatchStepThreads / 4 charges.  A replica's application items become ready
// when its field segments and deposition items have all finished, its gather
// items when its application items have; counts per replica say so.  Nothing
// waits on a grid-wide barrier: while some CTAs stream field segments, others
// deposit, apply and gather the replicas whose fields were just written
// (still in L2).
constexpr int kBatchStepThreads = 256;
constexpr int kBatchChunksPerItem = 2;
enum : int { kItemField = 0, kItemDeposit = 1, kItemApply = 2, kItemGather = 3 };
struct BatchItem {
  int rep;
  int a, b, c, d;  // field: y0, rows, za, zb; deposition: item index in the replica
};
// queue claims and the launch count; counts only grow (the bases move to the
// claims reached by the end of each launch), so nothing is reset between
// launches
struct BatchSched {
  unsigned long long epoch;     // launches completed
  unsigned long long next[2];   // claims made on the field and deposition queues
  unsigned long long base[2];   // claims made before this launch
  unsigned long long exits;     // CTAs that have left a launch
  unsigned int err;             // kErrTimeout when a wait ran out
  unsigned int pad;
};
// one replica: items of each kind finished (grows by its item count every
// launch), and claims of its application and gather items with their values
// at the start of this launch
struct RepSync {
  unsigned long long done[4];
  unsigned long long claim[2];
  unsigned long long base[2];
};
struct BatchStepArgs {
  const RepDesc* desc;
  int nrep;
  const BatchItem* q[2];  // field and deposition items
  int n[2];
  BatchSched* sched;
  RepSync* sync;
  int par;
  int thermo;
  double gamma, kT;
  int field_ctas;          // CTAs [0, field_ctas) start with field items, the rest with
                           // particle work; all take field items once theirs run out
  unsigned long long wait_ns;  // bound of a wait for dependent work
};
// dynamic shared memory of the kernel (that of the row tiles) and its CTAs
// per SM (0: it cannot run); the launch is cooperative with grid = CTAs per
// SM x SMs, so every CTA is resident together
size_t batch_step_smem();
int batch_step_occupancy(int prec);
cudaError_t launch_batch_step(int prec, const BatchStepArgs& a, int grid, cudaStream_t st);
// field update of every replica (memd_field.cu)
void launch_fused_batch(int prec, const RepDesc* desc, const int* cta_rep, int nctas, int par,
                        int ty, int pf, int tw, cudaStream_t st);
// the batch's host I/O block (memd_batch_step_io): the members' particles in
// order, member r from entry off[r] of ntot = off[count]; io_layout(ntot),
// with count error words at its err offset
inline int64_t batch_io_bytes(int64_t ntot, int count) {
  return io_layout(ntot).err + 4 * (((int64_t)count + 1) / 2) * 2;
}
void launch_io_unpack_batch(const RepDesc* desc, const int64_t* off, int count, int64_t ntot,
                            const void* io, cudaStream_t st);
void launch_io_pack_batch(const RepDesc* desc, const int64_t* off, int count, int64_t ntot,
                          void* io, cudaStream_t st, int part = kIoAll);
// particle kernels of every replica (memd_particles.cu); thermostat from the arguments
void launch_deposit_batch(const RepDesc* desc, const int* cta_rep, int nctas, int thermo,
                          double gamma, double kT, cudaStream_t st);
void launch_apply_batch(int prec, const RepDesc* desc, const int* cta_rep, int nctas, int par,
                        cudaStream_t st);
// one thread per charge (cta_rep over kWideThreads charges a CTA)
void launch_deposit_batch_wide(const RepDesc* desc, const int* cta_rep, int nctas,
                               cudaStream_t st);
void launch_gather_batch_wide(int prec, const RepDesc* desc, const int* cta_rep, int nctas,
                              int par, int thermo, cudaStream_t st);
// dense form: CTA b takes the kApplyChunk transfer words from chunk[b].y *
// kApplyChunk of replica chunk[b].x
constexpr int kApplyThreads = 256;
constexpr int kApplyPairs = 4;  // 16-byte word pairs a thread, all loaded before any store
constexpr int64_t kApplyChunk = 2 * kApplyPairs * kApplyThreads;  // words a CTA
void launch_apply_dense_batch(int prec, const RepDesc* desc, const int2* chunk, int nchunks,
                              int par, cudaStream_t st);
void launch_gather_batch(int prec, const RepDesc* desc, const int* cta_rep, int nctas, int par,
                         int thermo, double gamma, double kT, cudaStream_t st);
// per-particle constants: h = (dt/2)/m always; sig when thermo is set
void launch_particle_constants(const StepParams& sp, Particles p, cudaStream_t st);
// energy pieces into partial sums (memd_particles.cu)
void launch_particle_energy(const Mesh& m, const StepParams& sp, Particles p,
                            const double* ie64, double* part_ke, double* part_self,
                            cudaStream_t st);

// ------------------------------------------------------- field diagnostics
// (memd_field.cu)
void launch_field_energy(const Mesh& m, int prec, const void* D, const void* B,
                         const void* ie, double coefB, double* part_el, double* part_mag,
                         cudaStream_t st);
// partial sums (reduce_blocks() each) of E^2 over the 3V links, then of
// E_x, E_y, E_z over their V links, E = D / eps
void launch_field_moments(int prec, const void* D, const void* ie, int64_t V, double* part,
                          cudaStream_t st);
// Gauss check: mismatch count of div Lg vs Q and max |a^2 div D - Q 2^-48|
void launch_gauss_check(const Mesh& m, int prec, const void* D, const long long* Lg,
                        const long long* Q, double a2, double* part_res,
                        unsigned long long* mismatch, cudaStream_t st);

}  // namespace memd
