// memd_api.cu -- the C ABI of the MEMD library (declared in include/memd.h):
// context, device memory, the relaxation solver, the step sequence captured
// in a CUDA graph, and the state / diagnostic calls.  All arithmetic of the
// method runs in the kernels of memd_field.cu, memd_setup.cu and
// memd_particles.cu; this file only orders them.
#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <map>
#include <mutex>
#include <string>
#include <tuple>
#include <vector>

#include "memd.h"
#include "memd_ctx.cuh"
#include "memd_internal.cuh"

using namespace memd;

namespace {

const char* kStatusText[] = {"ok",
                             "invalid argument or state",
                             "Courant condition violated (c dt sqrt(3) >= a)",
                             "device allocation failed",
                             "CUDA error",
                             "a charge moved more than one cell in a step",
                             "Gauss ledger does not close",
                             "relaxation did not converge",
                             "dipole drift",
                             "timeout",
                             "call out of order",
                             "fixed-point overflow"};

memd_status fail(memd_ctx* c, memd_status s, const std::string& why) {
  if (c) c->last_error = why;
  return s;
}

#define CK(call)                                                                     \
  do {                                                                               \
    cudaError_t e_ = (call);                                                         \
    if (e_ != cudaSuccess)                                                           \
      return fail(c, MEMD_ERR_CUDA, std::string(#call) + ": " + cudaGetErrorString(e_)); \
  } while (0)

#define CKL()                                                                        \
  do {                                                                               \
    cudaError_t e_ = cudaGetLastError();                                             \
    if (e_ != cudaSuccess)                                                           \
      return fail(c, MEMD_ERR_CUDA, std::string("kernel launch: ") + cudaGetErrorString(e_)); \
  } while (0)

}  // namespace

void* memd_dalloc(memd_ctx* c, size_t bytes) {
  if (bytes < 256) bytes = 256;
  void* p = nullptr;
  if (c->alloc) {
    p = c->alloc(c->alloc_user, bytes, (void*)c->stream);
  } else if (cudaMalloc(&p, bytes) != cudaSuccess) {
    cudaGetLastError();
    p = nullptr;
  }
  if (p) c->blocks.emplace_back(p, bytes);
  return p;
}

void memd_dfree(memd_ctx* c, void* p) {
  if (!p) return;
  for (size_t i = 0; i < c->blocks.size(); ++i)
    if (c->blocks[i].first == p) {
      if (c->free_fn)
        c->free_fn(c->alloc_user, p, c->blocks[i].second, (void*)c->stream);
      else
        cudaFree(p);
      c->blocks.erase(c->blocks.begin() + i);
      return;
    }
}

namespace {

void* dalloc(memd_ctx* c, size_t bytes) { return memd_dalloc(c, bytes); }
void dfree(memd_ctx* c, void* p) { memd_dfree(c, p); }

}  // namespace

size_t memd_esz(const memd_ctx* c) { return c->prec == MEMD_FP32 ? sizeof(float) : sizeof(double); }

StepParams memd_step_params(const memd_ctx* c, int thermo, double gamma, double kT) {
  StepParams sp{};
  sp.dt = c->dt;
  sp.coefB = c->dt / c->mesh.a;
  sp.coefD = c->c * c->c * c->dt / c->mesh.a;
  sp.scale = std::ldexp(1.0, -48) / (c->mesh.a * c->mesh.a);
  sp.Vbox = c->Vbox;
  sp.inv_V = 1.0 / c->Vbox;
  sp.self_pre = 0.5 / (c->mesh.a * c->mesh.a);
  sp.dip_unit = c->mesh.a / (double)kS;
  for (int t = 0; t < 8; ++t) sp.G[t] = c->G[t];
  for (int t = 0; t < 9; ++t) sp.Minv[t] = c->Minv[t];
  for (int t = 0; t < 9; ++t) sp.Mdip[t] = c->Minv[t] * sp.dip_unit * sp.inv_V;
  for (int t = 0; t < 8; ++t) sp.Gf[t] = (float)sp.G[t];
  for (int t = 0; t < 9; ++t) sp.Mdipf[t] = (float)sp.Mdip[t];
  sp.self_pref = (float)sp.self_pre;
  sp.self_mode = c->self_mode;
  sp.dipole_corr = c->dipole_corr;
  sp.thermo = thermo;
  sp.gamma = gamma;
  sp.kT = kT;
  sp.seed = c->seed;
  sp.wait_ns = c->wait_ns;
  return sp;
}

namespace {

size_t esz(const memd_ctx* c) { return memd_esz(c); }
StepParams step_params(const memd_ctx* c, int thermo, double gamma, double kT) {
  return memd_step_params(c, thermo, gamma, kT);
}

}  // namespace

memd_status memd_check_err(memd_ctx* c) {
  unsigned int err = 0;
  CK(cudaMemcpyAsync(&err, &c->ds->err, sizeof(err), cudaMemcpyDeviceToHost, c->stream));
  CK(cudaStreamSynchronize(c->stream));
  if (err) {
    CK(cudaMemsetAsync(&c->ds->err, 0, sizeof(unsigned int), c->stream));
    if (err & kErrTimeout)  // a grid barrier gave up: start its words afresh
      CK(cudaMemsetAsync(&c->ds->bar_arrivals, 0, sizeof(unsigned long long), c->stream));
    CK(cudaStreamSynchronize(c->stream));
    if (err & kErrCellJump) return fail(c, MEMD_ERR_CELL_JUMP, "a charge moved more than one cell");
    if (err & kErrGauss) return fail(c, MEMD_ERR_GAUSS, "Gauss scan did not close (system not neutral)");
    if (err & kErrNonFinite) return fail(c, MEMD_ERR_INVALID, "non-finite or out-of-range input");
    if (err & kErrTimeout) return fail(c, MEMD_ERR_TIMEOUT, "a bounded wait in a kernel gave up");
    return fail(c, MEMD_ERR_OVERFLOW, "fixed-point overflow");
  }
  return MEMD_OK;
}

namespace {

memd_status check_err(memd_ctx* c) { return memd_check_err(c); }

// scalar slots in c->red after the partial arrays
enum {
  kS_PW = 0, kS_RZ0 = 1, kS_RZ1 = 2, kS_RES = 3, kS_EMAX = 4, kS_A = 5, kS_B = 6, kS_C = 7,
  kS_RMAX = 13, kS_DONE = 14, kS_TOL = 15
};

void harvest_timing(memd_ctx* c) {
  if (!c->timing_pending) return;
  float ms = 0;
  if (cudaEventSynchronize(c->ev1) == cudaSuccess &&
      cudaEventElapsedTime(&ms, c->ev0, c->ev1) == cudaSuccess) {
    c->field_ms += ms;
    c->field_launches += 1;
  }
  cudaGetLastError();
  c->timing_pending = false;
}

void drop_graphs(memd_ctx* c) {
  for (int t = 0; t < 2; ++t) {
    if (c->graph[t]) {
      cudaGraphExecDestroy(c->graph[t]);
      c->graph[t] = nullptr;
    }
    if (c->io_graph[t]) {
      cudaGraphExecDestroy(c->io_graph[t]);
      c->io_graph[t] = nullptr;
    }
  }
}

double* scal(memd_ctx* c) { return c->red + 4 * reduce_blocks(); }

// the ledger between a component-major host array of 3 V words (link (d, v)
// at d V + v) and its vertex-major words on the device: one strided copy a
// component
cudaError_t ledger_to_host(memd_ctx* c, void* host, cudaStream_t st) {
  const int64_t V = c->mesh.V;
  for (int d = 0; d < 3; ++d) {
    const cudaError_t e =
        cudaMemcpy2DAsync((long long*)host + d * V, 8, c->Lg + kLT * tl_pair(d, 0), 3 * kLT * 8, 8,
                          (size_t)V, cudaMemcpyDeviceToHost, st);
    if (e != cudaSuccess) return e;
  }
  return cudaSuccess;
}
cudaError_t ledger_from_host(memd_ctx* c, const void* host, cudaStream_t st) {
  const int64_t V = c->mesh.V;
  for (int d = 0; d < 3; ++d) {
    const cudaError_t e =
        cudaMemcpy2DAsync(c->Lg + kLT * tl_pair(d, 0), 3 * kLT * 8, (const long long*)host + d * V,
                          8, 8, (size_t)V, cudaMemcpyHostToDevice, st);
    if (e != cudaSuccess) return e;
  }
  return cudaSuccess;
}

// zero the transfer words (every kLT-th word) of a buffer, leaving the
// ledger words between them
cudaError_t clear_transfers(memd_ctx* c, long long* T, cudaStream_t st) {
  launch_clear_transfers(T, 3 * c->mesh.V, st);
  return cudaGetLastError();
}

}  // namespace

// ------------------------------------------------------------------ relaxation
// Sec. II: energy minimisation of sum D^2 / 2 eps over divergence-free
// changes of D, i.e. curl E = 0, by preconditioned conjugate gradients on
// plaquette rotations theta: D = D0 + C^T theta, gradient -C(ie D), Jacobi
// preconditioner sum of ie around each plaquette.  It keeps div D and the
// mean of D exactly (up to rounding).  FP64 throughout.
namespace {

// After the recursive residual meets the tolerance the iteration freezes
// (kS_DONE): continuing in round-off would divide noise by noise.  The host
// then checks the true residual and restarts from it if needed.
__global__ void k_pcg_dir(int64_t n, double* __restrict__ p, const double* __restrict__ z,
                          double* __restrict__ sc, int rz_new, int rz_old, int first) {
  const int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (first) {
    if (t < n) p[t] = z[t];
    return;
  }
  if (sc[kS_DONE] != 0.0) return;
  if (sc[kS_RMAX] <= sc[kS_TOL] * sc[kS_EMAX]) {
    if (t == 0) sc[kS_DONE] = 1.0;
    return;
  }
  if (t >= n) return;
  const double a = sc[rz_new], b = sc[rz_old];
  const double beta = (b != 0.0) ? a / b : 0.0;
  p[t] = z[t] + beta * p[t];
}

__global__ void k_set_scalar(double* sc, int slot, double v) {
  if (threadIdx.x == 0 && blockIdx.x == 0) sc[slot] = v;
}

__global__ void k_div(int64_t n, double* __restrict__ z, const double* __restrict__ r,
                      const double* __restrict__ diag) {
  const int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (t < n) z[t] = r[t] / diag[t];
}

__global__ void k_fill_unit(int64_t V, double* __restrict__ D, int d) {
  const int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (t < 3 * V) D[t] = (t / V == d) ? 1.0 : 0.0;
}

inline unsigned nb(int64_t n) { return (unsigned)((n + 255) / 256); }

}  // namespace

// inverse of a 3 x 3 matrix (row major); false if singular
static bool invert3(const double a[9], double out[9]) {
  const double c00 = a[4] * a[8] - a[5] * a[7], c01 = a[5] * a[6] - a[3] * a[8],
               c02 = a[3] * a[7] - a[4] * a[6];
  const double det = a[0] * c00 + a[1] * c01 + a[2] * c02;
  if (!(std::fabs(det) > 0.0)) return false;
  const double id = 1.0 / det;
  out[0] = c00 * id;
  out[1] = (a[2] * a[7] - a[1] * a[8]) * id;
  out[2] = (a[1] * a[5] - a[2] * a[4]) * id;
  out[3] = c01 * id;
  out[4] = (a[0] * a[8] - a[2] * a[6]) * id;
  out[5] = (a[2] * a[3] - a[0] * a[5]) * id;
  out[6] = c02 * id;
  out[7] = (a[1] * a[6] - a[0] * a[7]) * id;
  out[8] = (a[0] * a[4] - a[1] * a[3]) * id;
  return true;
}

static memd_status relax(memd_ctx* c, double* D64, double tol, int maxit) {
  const Mesh& m = c->mesh;
  const int64_t n = 3 * m.V;
  const cudaStream_t st = c->stream;
  double* buf = (double*)dalloc(c, sizeof(double) * 6 * n);
  if (!buf) return fail(c, MEMD_ERR_OOM, "relaxation scratch");
  double *r = buf, *z = buf + n, *p = buf + 2 * n, *u = buf + 3 * n, *w = buf + 4 * n,
         *diag = buf + 5 * n;
  double* part = c->red;
  double* sc = scal(c);
  const int R = reduce_blocks();
  launch_plaquette_diag(m, diag, c->ie64, st);
  // true residual max|circ(ie D)| and max|ie D|; ok when res <= tol * emax
  auto check = [&](bool& ok, bool& frozen) -> memd_status {
    launch_circ64(m, w, D64, c->ie64, -1.0, st);
    launch_absmax(w, nullptr, n, part, st);
    launch_finish(part, 1, sc + kS_RES, st);
    launch_absmax(D64, c->ie64, n, part, st);
    launch_finish(part, 1, sc + kS_EMAX, st);
    double h[2], done = 0;
    CK(cudaMemcpyAsync(h, sc + kS_RES, 2 * sizeof(double), cudaMemcpyDeviceToHost, st));
    CK(cudaMemcpyAsync(&done, sc + kS_DONE, sizeof(double), cudaMemcpyDeviceToHost, st));
    CK(cudaStreamSynchronize(st));
    ok = h[0] <= tol * h[1];
    frozen = done != 0.0;
    return MEMD_OK;
  };
  // (re)start from the true residual held in w
  auto restart = [&]() {
    cudaMemcpyAsync(r, w, n * sizeof(double), cudaMemcpyDeviceToDevice, st);
    k_div<<<nb(n), 256, 0, st>>>(n, z, r, diag);
    k_pcg_dir<<<nb(n), 256, 0, st>>>(n, p, z, sc, 0, 0, 1);
    launch_dot(r, z, n, part, st);
    launch_finish(part, 0, sc + kS_RZ0, st);
    k_set_scalar<<<1, 32, 0, st>>>(sc, kS_DONE, 0.0);
    k_set_scalar<<<1, 32, 0, st>>>(sc, kS_TOL, 0.5 * tol);
  };
  // kChunk iterations (an even count, so that the r.z slots are back in
  // place) between checks of the true residual; the chunk is captured once
  // as a CUDA graph and replayed, or launched directly if capture fails
  constexpr int kChunk = 24;
  auto chunk = [&]() {
    for (int j = 0; j < kChunk; ++j) {
      const int parity = j & 1;
      const int old_slot = kS_RZ0 + parity, new_slot = kS_RZ0 + (parity ^ 1);
      // four launches per iteration: transpose map, operator with p.w,
      // update with r.z and max|r|, direction (see memd_field.cu)
      launch_curlT64(m, u, p, st);
      launch_cg_apply(m, w, u, c->ie64, p, part, st);
      launch_cg_update(n, D64, u, r, w, z, diag, part, sc, old_slot, part + R, part + 2 * R, st);
      launch_cg_direction(n, p, z, sc, part + R, part + 2 * R, new_slot, old_slot, st);
    }
  };
  cudaGraphExec_t gexec = nullptr;
  bool ok = false, frozen = false;
  k_set_scalar<<<1, 32, 0, st>>>(sc, kS_DONE, 0.0);
  memd_status s = check(ok, frozen);
  int it = 0;
  if (s == MEMD_OK && !ok) {
    restart();
    if (c->use_graphs) {
      cudaGraph_t g = nullptr;
      if (cudaStreamBeginCapture(st, cudaStreamCaptureModeThreadLocal) == cudaSuccess) {
        chunk();
        if (cudaStreamEndCapture(st, &g) != cudaSuccess ||
            cudaGraphInstantiate(&gexec, g, 0) != cudaSuccess)
          gexec = nullptr;
        if (g) cudaGraphDestroy(g);
      }
      cudaGetLastError();
    }
    while (it < maxit) {
      if (gexec) {
        if (cudaGraphLaunch(gexec, st) != cudaSuccess) {
          s = fail(c, MEMD_ERR_CUDA, "relaxation graph launch");
          break;
        }
      } else {
        chunk();
      }
      it += kChunk;
      if (cudaGetLastError() != cudaSuccess) {
        s = fail(c, MEMD_ERR_CUDA, "relaxation kernel launch");
        break;
      }
      s = check(ok, frozen);
      if (s != MEMD_OK || ok) break;
      if (frozen) restart();  // the recursion converged but the true residual did not
    }
  }
  if (gexec) cudaGraphExecDestroy(gexec);
  c->relax_iters_last = it;
  dfree(c, buf);
  if (s != MEMD_OK) return s;
  if (!ok) return fail(c, MEMD_ERR_RELAX_NOCONV, "relaxation did not reach its tolerance");
  return MEMD_OK;
}

// the fused field update of buffer parity par with the context's kernel choice
// The row kernel for this context alone: a one-entry descriptor table
// (buffers by absolute parity) and the work split over a persistent grid.
// False when the mesh does not fit the kernel (x extent not a multiple of
// the vector width, buffers not 16-byte aligned) or memory is short.
static bool rows_setup(memd_ctx* c, int nt) {
  if (c->rows_nt == nt && c->rows_desc) return true;
  dfree(c, c->rows_desc);
  dfree(c, c->rows_segs);
  dfree(c, c->rows_first);
  c->rows_desc = nullptr;
  c->rows_segs = nullptr;
  c->rows_first = nullptr;
  c->rows_nt = 0;
  int sms = 0;
  if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, c->device) != cudaSuccess)
    return false;
  const int occ = rows_occupancy(c->prec, nt);
  std::vector<RowSeg> segs;
  std::vector<int> first;
  if (occ <= 0 || !rows_plan(std::vector<memd_ctx*>{c}, c->prec, nt, occ * sms, segs, first))
    return false;
  RepDesc d;
  std::memset(&d, 0, sizeof(d));
  d.m = c->mesh;
  d.sp = step_params(c, 0, 0.0, 0.0);
  for (int k = 0; k < 2; ++k) {
    d.D[k] = c->Dbuf[k];
    d.B[k] = c->Bbuf[k];
  }
  d.ie = c->ie;
  c->rows_desc = (RepDesc*)dalloc(c, sizeof(RepDesc));
  c->rows_segs = (RowSeg*)dalloc(c, sizeof(RowSeg) * std::max<size_t>(1, segs.size()));
  c->rows_first = (int*)dalloc(c, sizeof(int) * first.size());
  if (!c->rows_desc || !c->rows_segs || !c->rows_first ||
      cudaMemcpyAsync(c->rows_desc, &d, sizeof(d), cudaMemcpyHostToDevice, c->stream) !=
          cudaSuccess ||
      cudaMemcpyAsync(c->rows_segs, segs.data(), sizeof(RowSeg) * segs.size(),
                      cudaMemcpyHostToDevice, c->stream) != cudaSuccess ||
      cudaMemcpyAsync(c->rows_first, first.data(), sizeof(int) * first.size(),
                      cudaMemcpyHostToDevice, c->stream) != cudaSuccess ||
      cudaStreamSynchronize(c->stream) != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  c->rows_nctas = occ * sms;
  c->rows_nt = nt;
  return true;
}

static void launch_field(memd_ctx* c, int par, double cB, double cD, FusedCfg cfg) {
  if (cfg.rows)
    launch_rows_batch(c->prec, c->rows_desc, c->rows_segs, c->rows_first, c->rows_nctas,
                      cfg.rows, par, c->stream);
  else if (cfg.tma)
    launch_fused_tma(c->mesh, c->prec, c->tma, par, c->Dbuf[par], c->Bbuf[par], c->ie,
                     c->Dbuf[par ^ 1], c->Bbuf[par ^ 1], cB, cD, cfg, &c->ds->err, c->stream);
  else
    launch_fused_curl(c->mesh, c->prec, c->Dbuf[par], c->Bbuf[par], c->ie, c->Dbuf[par ^ 1],
                      c->Bbuf[par ^ 1], cB, cD, cfg, c->stream);
}

// ------------------------------------------------------------------ autotuner
// Picks the field kernel (halo-loop, one-thread-per-site with its prefetch
// depth, or TMA-staged), its tile height and z-chunk for this mesh by timing
// every candidate on the context's own buffers (median of 3 samples of 1 to
// 20 back-to-back launches, after one warm-up).  Results are cached per mesh
// shape, precision and kernel choice for the life of the process.
static memd_status autotune_fused(memd_ctx* c) {
  memd::NvtxRange nvtx_("autotune_fused");
  static std::mutex mu;
  static std::map<std::tuple<int, int, int, int, int>, FusedCfg> cache;
  c->tma_ok = (c->field_kernel == MEMD_FIELD_AUTO || c->field_kernel == MEMD_FIELD_TMA) &&
              tma_supported(c->mesh, c->prec) &&
              tma_make_maps(c->mesh, c->prec, c->Dbuf, c->Bbuf, c->ie, &c->tma);
  {
    // a shape fixed at create is taken as it is (checked there); the row
    // kernel falls back to the default site shape where the mesh does not fit
    const int* fs = c->field_shape;
    if (fs[0] || fs[3]) {
      FusedCfg f = fused_default(c->mesh);
      if (fs[3]) {
        if (rows_setup(c, fs[3])) {
          f.rows = fs[3];
        } else {
          f.site = 1;
        }
      } else {
        f.ty = fs[0];
        f.zchunk = std::min(fs[1], c->mesh.n[2]);
        f.site = c->field_kernel == MEMD_FIELD_SITE ? fs[2] : 0;
        f.tma = c->field_kernel == MEMD_FIELD_TMA && c->tma_ok ? 1 : 0;
      }
      c->fcfg = f;
      return MEMD_OK;
    }
  }
  const auto key = std::make_tuple(c->mesh.n[0], c->mesh.n[1], c->mesh.n[2], c->prec,
                                   c->field_kernel * 2 + (c->tma_ok ? 1 : 0));
  {
    std::lock_guard<std::mutex> g(mu);
    auto it = cache.find(key);
    if (it != cache.end() && (it->second.rows == 0 || rows_setup(c, it->second.rows))) {
      c->fcfg = it->second;
      return MEMD_OK;
    }
  }
  FusedCfg cand[160];
  int nc = 0;
  const int fk = c->field_kernel;
  // Left to choose, the row kernel's two widths are the only candidates
  // where the mesh fits it: in the step the field pass runs beside the
  // deposition, and there the row kernel was the fastest measured on every
  // such mesh (64^3 salt and colloid systems: 35.2 / 31.2 us a step against
  // 36-39 / 33-35 for the tile kernels that time fastest alone; 256^3: the
  // row kernel is also the fastest alone), while the tile kernels' timings
  // alone do not carry over to the step.
  const bool rows_only = fk == MEMD_FIELD_AUTO && rows_setup(c, 256);
  const bool want_ldg = !rows_only && (fk == MEMD_FIELD_AUTO || fk == MEMD_FIELD_LDG ||
                                       (fk == MEMD_FIELD_TMA && !c->tma_ok));
  const bool want_site = !rows_only && (fk == MEMD_FIELD_AUTO || fk == MEMD_FIELD_SITE);
  if (want_ldg) nc = fused_candidates(c->mesh, c->prec, cand, 32);
  if (want_site) {
    // the one-thread-per-site plain-load kernel, same tile shapes, loads 1 or
    // 2 planes ahead
    for (int pf = 1; pf <= 2; ++pf) {
      FusedCfg t[32];
      const int nt = fused_candidates(c->mesh, c->prec, t, 32);
      for (int i = 0; i < nt; ++i) {
        if (pf > 1 && t[i].zchunk < 4) continue;  // too few planes to run ahead
        t[i].site = pf;
        cand[nc++] = t[i];
      }
    }
  }
  if (c->tma_ok && !rows_only) {
    FusedCfg t[32];
    const int nt = fused_candidates(c->mesh, 1, t, 32);  // the TMA kernel has all three heights
    for (int i = 0; i < nt && nc < 158; ++i) {
      t[i].tma = 1;
      cand[nc++] = t[i];
    }
  }
  // the row kernel (whole rows of 16-byte vectors), where the mesh fits it;
  // asked for alone and not fitting, the site kernel's shapes stand in
  if (fk == MEMD_FIELD_AUTO || fk == MEMD_FIELD_ROWS) {
    const bool fits = rows_setup(c, 256);
    for (int nt = 256; nt <= 512 && fits; nt *= 2) {
      FusedCfg r = fused_default(c->mesh);
      r.tma = 0;
      r.site = 0;
      r.rows = nt;
      cand[nc++] = r;
    }
    if (fk == MEMD_FIELD_ROWS && !fits) {
      for (int pf = 1; pf <= 2; ++pf) {
        FusedCfg t[32];
        const int nt2 = fused_candidates(c->mesh, c->prec, t, 32);
        for (int i = 0; i < nt2 && nc < 160; ++i) {
          if (pf > 1 && t[i].zchunk < 4) continue;
          t[i].site = pf;
          cand[nc++] = t[i];
        }
      }
    }
  }
  cudaEvent_t e0, e1;
  CK(cudaEventCreate(&e0));
  CK(cudaEventCreate(&e1));
  float best = 1e30f;
  FusedCfg pick = fused_default(c->mesh);
  // launches per timing sample: small meshes take a few microseconds a
  // launch, so one launch between two events would time mostly the events
  const int reps = c->mesh.V <= (1 << 16) ? 20 : (c->mesh.V <= (1 << 20) ? 5 : 1);
  bool tma_checked = false;
  for (int i = 0; i < nc; ++i) {
    float t[3];
    // reads the current parity, writes a copy of it into the other one
    auto run = [&]() { launch_field(c, c->cur, 0.0, 0.0, cand[i]); };
    if (cand[i].tma && !c->tma_ok) continue;
    if (cand[i].rows && !rows_setup(c, cand[i].rows)) continue;
    run();
    if (cand[i].tma && !tma_checked) {
      // the first TMA launch runs alone: if any of its bounded waits gave up,
      // the TMA kernel is dropped for this context
      tma_checked = true;
      CK(cudaStreamSynchronize(c->stream));
      unsigned int e = 0;
      CK(cudaMemcpy(&e, &c->ds->err, sizeof(e), cudaMemcpyDeviceToHost));
      if (e) {
        CK(cudaMemset(&c->ds->err, 0, sizeof(unsigned int)));
        c->tma_ok = false;
        continue;
      }
    }
    for (int r = 0; r < 3; ++r) {
      CK(cudaEventRecord(e0, c->stream));
      for (int k = 0; k < reps; ++k) run();
      CK(cudaEventRecord(e1, c->stream));
      CK(cudaEventSynchronize(e1));
      CK(cudaEventElapsedTime(&t[r], e0, e1));
    }
    CKL();
    const float med = std::max(std::min(t[0], t[1]), std::min(std::max(t[0], t[1]), t[2]));
    if (med < best) {
      best = med;
      pick = cand[i];
    }
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  {
    const memd_status e = check_err(c);
    if (e != MEMD_OK) return e;
  }
  if (pick.rows && !rows_setup(c, pick.rows)) pick = fused_default(c->mesh);
  c->fcfg = pick;
  std::lock_guard<std::mutex> g(mu);
  cache[key] = pick;
  return MEMD_OK;
}

// ----------------------------------------------------------------- public API
extern "C" {

void memd_default_options(memd_options* o) {
  if (!o) return;
  std::memset(o, 0, sizeof(*o));
  o->precision = MEMD_FP64;
  o->self_mode = MEMD_SELF_GF;
  o->dipole_corr = 1;
  o->relax_max_iter = 200000;
  o->relax_tol = 1e-12;
  o->seed = 0;
  o->cuda_stream = nullptr;
  o->device = -1;
  o->use_graphs = 1;
}

const char* memd_status_string(memd_status s) {
  int i = (int)s;
  if (i < 0 || i > 11) return "unknown status";
  return kStatusText[i];
}

const char* memd_last_error(const memd_ctx* c) {
  if (!c) return "no context";
  return c->last_error.c_str();
}

void memd_destroy(memd_ctx* c) {
  if (!c) return;
  cudaSetDevice(c->device);
  if (c->stream) cudaStreamSynchronize(c->stream);
  drop_graphs(c);
  if (c->ev0) cudaEventDestroy(c->ev0);
  if (c->ev1) cudaEventDestroy(c->ev1);
  if (c->fork) cudaEventDestroy(c->fork);
  if (c->join) cudaEventDestroy(c->join);
  if (c->side) cudaStreamDestroy(c->side);
  if (c->err_host) cudaFreeHost(c->err_host);
  if (c->io_host) cudaFreeHost(c->io_host);
  while (!c->blocks.empty()) dfree(c, c->blocks.back().first);
  if (c->own_stream && c->stream) cudaStreamDestroy(c->stream);
  delete c;
}

// the profile's parameters against the box (Sec. II; the interface kinds
// need their interface inside the box)
static bool eps_valid(const memd_eps_profile* e, const double box[3], double a) {
  const double* p = e->params;
  const bool axis_ok = e->axis >= 0 && e->axis <= 2;
  auto pos = [](double x) { return x > 0.0 && std::isfinite(x); };
  switch (e->kind) {
    case MEMD_EPS_CONST:
      return true;
    case MEMD_EPS_LINKS:
    case MEMD_EPS_CUT:
      return e->values != nullptr;
    case MEMD_EPS_VERTICES:
      return e->values != nullptr && p[0] >= 0.0 && std::isfinite(p[0]);
    case MEMD_EPS_TANH:
    case MEMD_EPS_SIN:
      return axis_ok;
    case MEMD_EPS_PLANES:
      return axis_ok && pos(p[0]) && pos(p[1]) && p[2] >= 0.0 && p[2] <= p[3] &&
             p[3] < box[e->axis];
    case MEMD_EPS_SPHERE:
      if (!pos(p[0]) || !pos(p[1]) || !pos(p[5])) return false;
      for (int d = 0; d < 3; ++d)
        if (!std::isfinite(p[2 + d]) || !(p[5] + a < 0.5 * box[d])) return false;
      return true;
    default:
      return false;
  }
}

// Permittivity on the links (Sec. II, Fig. 2b, Eq. dielectric-interpolation)
// and the effective tensor (Sec. V): first through the three cell problems
// of the scalar potential; if that solver does not converge, by relaxing a
// charge-free field of mean D = e_d, whose mean E is then column d of
// eps_eff^-1.  A context that already had a permittivity gets it back, with
// its potentials and tensor, when any step fails.
// map a profile onto the links and form the effective tensor; dev_values:
// the profile's values already on the device (else eps->values is copied)
static memd_status setup_eps(memd_ctx* c, const memd_eps_profile* eps,
                             const double* dev_values = nullptr) {
  const cudaStream_t st = c->stream;
  const int64_t V = c->mesh.V;
  const size_t n3 = 3 * (size_t)V;
  const bool had = c->eps_ready;
  memd_status s = MEMD_OK;
  double *vals = nullptr, *save = nullptr, *psi = nullptr, *D64 = nullptr;
  double M[9];
  bool mapped = false;
  EpsDesc e{};
  e.kind = eps->kind;
  e.axis = eps->axis;
  for (int t = 0; t < 8; ++t) e.p[t] = eps->params[t];
  const size_t cnt = eps->kind == MEMD_EPS_LINKS      ? n3
                     : eps->kind == MEMD_EPS_VERTICES ? (size_t)V
                     : eps->kind == MEMD_EPS_CUT      ? 4 * (size_t)V
                                                      : 0;
  if (cnt && !dev_values) {
    vals = (double*)dalloc(c, cnt * sizeof(double));
    if (!vals) {
      s = fail(c, MEMD_ERR_OOM, "eps values");
      goto out;
    }
    if (cudaMemcpyAsync(vals, eps->values, cnt * sizeof(double), cudaMemcpyHostToDevice, st) !=
        cudaSuccess) {
      s = fail(c, MEMD_ERR_CUDA, "eps upload");
      goto out;
    }
  }
  if (had) {
    save = (double*)dalloc(c, n3 * sizeof(double));
    if (!save) {
      s = fail(c, MEMD_ERR_OOM, "eps save");
      goto out;
    }
    if (cudaMemcpyAsync(save, c->ie64, n3 * sizeof(double), cudaMemcpyDeviceToDevice, st) !=
        cudaSuccess) {
      s = fail(c, MEMD_ERR_CUDA, "eps save");
      goto out;
    }
  }
  launch_eps_links(c->mesh, e, dev_values ? dev_values : vals, c->ie64, &c->ds->err, st);
  launch_cast(c->prec, c->ie, c->ie64, (int64_t)n3, st);
  mapped = true;
  if (cudaGetLastError() != cudaSuccess) {
    s = fail(c, MEMD_ERR_CUDA, "eps kernels");
    goto out;
  }
  s = check_err(c);
  if (s != MEMD_OK) goto out;
  psi = (double*)dalloc(c, n3 * sizeof(double));
  if (psi) {
    double ef[9];
    const memd_status ms =
        mg_eps_eff(c, psi, ef, std::min(c->relax_tol, 1e-12), c->relax_maxit);
    if (ms == MEMD_OK && invert3(ef, M)) goto tensor;
    dfree(c, psi);
    psi = nullptr;
    cudaGetLastError();
  }
  D64 = (double*)dalloc(c, n3 * sizeof(double));
  if (!D64) {
    s = fail(c, MEMD_ERR_OOM, "relaxation field");
    goto out;
  }
  for (int d = 0; d < 3; ++d) {
    k_fill_unit<<<nb(n3), 256, 0, st>>>(V, D64, d);
    s = relax(c, D64, c->relax_tol, c->relax_maxit);
    if (s != MEMD_OK) goto out;
    for (int e2 = 0; e2 < 3; ++e2) {
      launch_dot(D64 + e2 * V, c->ie64 + e2 * V, V, c->red, st);
      launch_finish(c->red, 0, scal(c) + kS_A + e2, st);
    }
    double h[3];
    if (cudaMemcpyAsync(h, scal(c) + kS_A, 3 * sizeof(double), cudaMemcpyDeviceToHost, st) !=
            cudaSuccess ||
        cudaStreamSynchronize(st) != cudaSuccess) {
      s = fail(c, MEMD_ERR_CUDA, "eps_eff download");
      goto out;
    }
    for (int e2 = 0; e2 < 3; ++e2) M[3 * e2 + d] = h[e2] / (double)V;
  }
tensor:
  for (int t = 0; t < 9; ++t) c->eps_eff_inv[t] = M[t];
  for (int e2 = 0; e2 < 3; ++e2)
    for (int d = 0; d < 3; ++d) c->Minv[3 * e2 + d] = 0.5 * (M[3 * e2 + d] + M[3 * d + e2]);
  dfree(c, c->psi);
  c->psi = psi;
  psi = nullptr;
  c->eps_ready = true;
out:
  if (s != MEMD_OK && had && mapped) {
    cudaMemcpyAsync(c->ie64, save, n3 * sizeof(double), cudaMemcpyDeviceToDevice, st);
    launch_cast(c->prec, c->ie, c->ie64, (int64_t)n3, st);
    cudaStreamSynchronize(st);
  }
  dfree(c, vals);
  dfree(c, save);
  dfree(c, psi);
  dfree(c, D64);
  return s;
}

memd_status memd_create(const int32_t mesh[3], const double box[3], const memd_eps_profile* eps,
                        double c_light, double dt, const memd_options* opt, memd_ctx** out) {
  memd::NvtxRange nvtx_("memd_create");
  if (!out) return MEMD_ERR_INVALID;
  *out = nullptr;
  if (!mesh || !box || !eps) return MEMD_ERR_INVALID;
  memd_options o;
  if (opt)
    o = *opt;
  else
    memd_default_options(&o);
  for (int d = 0; d < 3; ++d)
    if (mesh[d] < 2 || !(box[d] > 0.0)) return MEMD_ERR_INVALID;
  const double a = box[0] / mesh[0];
  for (int d = 1; d < 3; ++d)
    if (std::fabs(box[d] / mesh[d] - a) > 1e-12 * a) return MEMD_ERR_INVALID;
  const int64_t V = (int64_t)mesh[0] * mesh[1] * mesh[2];
  if (3 * V >= (int64_t(1) << 31)) return MEMD_ERR_INVALID;
  if (!(c_light > 0.0) || !(dt > 0.0)) return MEMD_ERR_INVALID;
  if (!(c_light * dt * std::sqrt(3.0) < a)) return MEMD_ERR_COURANT;
  if (o.precision != MEMD_FP32 && o.precision != MEMD_FP64) return MEMD_ERR_INVALID;
  if (o.self_mode < 0 || o.self_mode > 2) return MEMD_ERR_INVALID;
  if (o.field_kernel < MEMD_FIELD_AUTO || o.field_kernel > MEMD_FIELD_ROWS) return MEMD_ERR_INVALID;
  if (o.step_engine < MEMD_STEP_AUTO || o.step_engine > MEMD_STEP_SINGLE) return MEMD_ERR_INVALID;
  if (o.apply_mode < MEMD_APPLY_AUTO || o.apply_mode > MEMD_APPLY_DENSE) return MEMD_ERR_INVALID;
  {
    // a fixed field-kernel shape: only the values its kernel uses, in range
    const int32_t* fs = o.field_shape;
    const bool any = fs[0] || fs[1] || fs[2] || fs[3];
    if (any) {
      const int fk = o.field_kernel;
      if (fk == MEMD_FIELD_AUTO) return MEMD_ERR_INVALID;
      if (fk == MEMD_FIELD_ROWS) {
        if (fs[0] || fs[1] || fs[2] || (fs[3] != 256 && fs[3] != 512)) return MEMD_ERR_INVALID;
      } else {
        if (fs[3] || (fs[0] != 4 && fs[0] != 8 && fs[0] != 16) || fs[1] < 1) return MEMD_ERR_INVALID;
        if (fs[0] == 16 && o.precision != MEMD_FP32) return MEMD_ERR_INVALID;
        if (fk == MEMD_FIELD_SITE ? (fs[2] != 1 && fs[2] != 2) : fs[2] != 0) return MEMD_ERR_INVALID;
      }
    }
  }
  if (!eps_valid(eps, box, a)) return MEMD_ERR_INVALID;

  memd_ctx* c = new memd_ctx();
  if (o.device >= 0) {
    c->device = o.device;
  } else if (cudaGetDevice(&c->device) != cudaSuccess) {
    delete c;
    return MEMD_ERR_CUDA;
  }
  if (cudaSetDevice(c->device) != cudaSuccess) {
    delete c;
    return MEMD_ERR_CUDA;
  }
  c->mesh.n[0] = mesh[0];
  c->mesh.n[1] = mesh[1];
  c->mesh.n[2] = mesh[2];
  c->mesh.V = V;
  c->mesh.a = a;
  for (int d = 0; d < 3; ++d) c->mesh.L[d] = box[d];
  {
    int ex = 0;
    c->mesh.a_pow2 = std::frexp(a, &ex) == 0.5 ? 1 : 0;
    c->mesh.inv_a = 1.0 / a;
    c->mesh.inv_aS = c->mesh.inv_a * (double)kS;
  }
  c->Vbox = box[0] * box[1] * box[2];
  c->c = c_light;
  c->dt = dt;
  c->prec = o.precision;
  c->self_mode = o.self_mode;
  c->dipole_corr = o.dipole_corr ? 1 : 0;
  c->relax_tol = o.relax_tol > 0 ? o.relax_tol : 1e-12;
  c->relax_maxit = o.relax_max_iter > 0 ? o.relax_max_iter : 200000;
  c->seed = o.seed;
  c->use_graphs = o.use_graphs;
  c->time_kernels = o.time_kernels;
  c->field_kernel = o.field_kernel;
  for (int k = 0; k < 4; ++k) c->field_shape[k] = o.field_shape[k];
  c->step_engine = o.step_engine;
  c->apply_mode = o.apply_mode;
  c->alloc = o.alloc;
  c->free_fn = o.free;
  c->alloc_user = o.alloc_user;
  if (o.cuda_stream) {
    c->stream = (cudaStream_t)o.cuda_stream;
  } else {
    if (cudaStreamCreateWithFlags(&c->stream, cudaStreamNonBlocking) != cudaSuccess) {
      delete c;
      return MEMD_ERR_CUDA;
    }
    c->own_stream = true;
  }
  memd_status s = MEMD_OK;
  const cudaStream_t st = c->stream;
  const size_t n3 = 3 * (size_t)V;
  for (int t = 0; t < 2; ++t) {
    c->Dbuf[t] = dalloc(c, n3 * esz(c));
    c->Bbuf[t] = dalloc(c, n3 * esz(c));
  }
  c->ie = dalloc(c, n3 * esz(c));
  c->ie64 = (double*)dalloc(c, n3 * sizeof(double));
  // transfer and ledger words interleaved (kLT): one block of 2 x 3V words
  c->Tb = (long long*)dalloc(c, kLT * n3 * sizeof(long long));
  c->Lg = c->Tb ? c->Tb + 1 : nullptr;
  c->ds = (DevState*)dalloc(c, sizeof(DevState));
  c->red = (double*)dalloc(c, sizeof(double) * (4 * reduce_blocks() + 32 + green_partials()));
  double* Gdev = nullptr;
  if (!c->Dbuf[0] || !c->Dbuf[1] || !c->Bbuf[0] || !c->Bbuf[1] || !c->ie || !c->ie64 ||
      !c->Lg || !c->Tb || !c->ds || !c->red) {
    s = fail(c, MEMD_ERR_OOM, "field allocation");
    goto done;
  }
  if (cudaMemsetAsync(c->ds, 0, sizeof(DevState), st) != cudaSuccess ||
      cudaMemsetAsync(c->Dbuf[0], 0, n3 * esz(c), st) != cudaSuccess ||
      cudaMemsetAsync(c->Dbuf[1], 0, n3 * esz(c), st) != cudaSuccess ||
      cudaMemsetAsync(c->Bbuf[0], 0, n3 * esz(c), st) != cudaSuccess ||
      cudaMemsetAsync(c->Bbuf[1], 0, n3 * esz(c), st) != cudaSuccess ||
      cudaMemsetAsync(c->Tb, 0, kLT * n3 * sizeof(long long), st) != cudaSuccess) {
    s = fail(c, MEMD_ERR_CUDA, "memset");
    goto done;
  }
  {
    // lattice Green's table (Sec. III)
    Gdev = c->red + 4 * reduce_blocks() + 32;
    launch_green(c->mesh, Gdev, scal(c) + 16, st);
    if (cudaGetLastError() != cudaSuccess) {
      s = fail(c, MEMD_ERR_CUDA, "setup kernels");
      goto done;
    }
    if (cudaMemcpyAsync(c->G, scal(c) + 16, 8 * sizeof(double), cudaMemcpyDeviceToHost, st) !=
        cudaSuccess) {
      s = fail(c, MEMD_ERR_CUDA, "green download");
      goto done;
    }
    s = setup_eps(c, eps);
    if (s != MEMD_OK) goto done;
  }
  if (cudaEventCreate(&c->ev0) != cudaSuccess || cudaEventCreate(&c->ev1) != cudaSuccess ||
      cudaEventCreateWithFlags(&c->fork, cudaEventDisableTiming) != cudaSuccess ||
      cudaEventCreateWithFlags(&c->join, cudaEventDisableTiming) != cudaSuccess ||
      cudaStreamCreateWithFlags(&c->side, cudaStreamNonBlocking) != cudaSuccess) {
    s = fail(c, MEMD_ERR_CUDA, "events");
    goto done;
  }
  // the field kernel is autotuned when a step first needs it (a system
  // stepped as one cooperative launch or only in batches never does)
  c->coop_grid = coop_grid(c->prec, c->device);
done:
  if (s != MEMD_OK) {
    memd_destroy(c);
    return s;
  }
  *out = c;
  return MEMD_OK;
}

static void free_particles(memd_ctx* c) {
  dfree(c, c->P.x);
  dfree(c, c->P.v);
  dfree(c, c->P.m);
  dfree(c, c->P.F);
  dfree(c, c->P.Ft);
  dfree(c, c->P.img);
  dfree(c, c->P.q);
  dfree(c, c->P.mv);
  dfree(c, c->P.h);
  dfree(c, c->P.sig);
  dfree(c, c->P.gm);
  dfree(c, c->pin);
  c->pin = nullptr;
  if (c->io_host) cudaFreeHost(c->io_host);
  dfree(c, c->io_dev);
  c->io_host = nullptr;
  c->io_dev = nullptr;
  c->io_n = -1;
  c->P = Particles{};
  c->sig_ready = false;
}

memd_status memd_init_field(memd_ctx* c, int64_t n, const double* pos, const int32_t* q,
                            const double* mass, const double* vel) {
  memd::NvtxRange nvtx_("memd_init_field");
  if (!c) return MEMD_ERR_INVALID;
  if (n < 0 || (n > 0 && (!pos || !q))) return fail(c, MEMD_ERR_INVALID, "bad particle arrays");
  CK(cudaSetDevice(c->device));
  const Mesh& m = c->mesh;
  const cudaStream_t st = c->stream;
  long long qtot = 0;
  for (int64_t p = 0; p < n; ++p) {
    if (q[p] > 32767 || q[p] < -32767) return fail(c, MEMD_ERR_INVALID, "valence out of range");
    qtot += q[p];
  }
  // the half kick divides by the mass
  if (mass)
    for (int64_t p = 0; p < n; ++p)
      if (!(mass[p] > 0.0) || !std::isfinite(mass[p]))
        return fail(c, MEMD_ERR_INVALID, "mass not positive and finite");
  // a non-neutral system gets a uniform background, exact in units e 2^-48
  const __int128 tot = (__int128)qtot * ((__int128)1 << 48);
  if (tot % m.V != 0)
    return fail(c, MEMD_ERR_INVALID, "non-neutral system needs an integer background per vertex");
  const long long bg = (long long)(tot / m.V);
  drop_graphs(c);
  harvest_timing(c);
  CK(cudaStreamSynchronize(st));
  free_particles(c);
  c->initialised = false;
  const size_t nn = (size_t)(n > 0 ? n : 1);
  c->P.n = n;
  c->P.x = (double*)dalloc(c, 3 * nn * sizeof(double));
  c->P.v = (double*)dalloc(c, 3 * nn * sizeof(double));
  c->P.m = (double*)dalloc(c, nn * sizeof(double));
  c->P.F = (double*)dalloc(c, 3 * nn * sizeof(double));
  c->P.Ft = (double*)dalloc(c, 3 * nn * sizeof(double));
  c->P.img = (int*)dalloc(c, 3 * nn * sizeof(int));
  c->P.q = (int*)dalloc(c, nn * sizeof(int));
  c->P.mv = (int*)dalloc(c, kMoveInts * nn * sizeof(int));
  c->P.h = (double*)dalloc(c, nn * sizeof(double));
  c->P.sig = (double*)dalloc(c, nn * sizeof(double));
  c->P.gm = (double*)dalloc(c, nn * sizeof(double));
  // staging of memd_set_particles (positions and images), kept with the particles
  c->pin = (double*)dalloc(c, 3 * nn * sizeof(double) + 3 * nn * sizeof(int));
  if (!c->P.x || !c->P.v || !c->P.m || !c->P.F || !c->P.Ft || !c->P.img || !c->P.q || !c->P.mv ||
      !c->P.h || !c->P.sig || !c->P.gm || !c->pin)
    return fail(c, MEMD_ERR_OOM, "particle allocation");
  double* pin = (double*)dalloc(c, 3 * nn * sizeof(double));
  long long* Q = (long long*)dalloc(c, sizeof(long long) * m.V);
  long long* scr = (long long*)dalloc(c, sizeof(long long) * scan_scratch(m));
  double* D64 = (double*)dalloc(c, sizeof(double) * 3 * m.V);
  memd_status s = MEMD_OK;
  if (!pin || !Q || !scr || !D64) {
    s = fail(c, MEMD_ERR_OOM, "init scratch");
  } else {
    std::vector<double> ones;
    if (n > 0) {
      CK(cudaMemcpyAsync(pin, pos, 3 * n * sizeof(double), cudaMemcpyHostToDevice, st));
      CK(cudaMemcpyAsync(c->P.q, q, n * sizeof(int), cudaMemcpyHostToDevice, st));
      if (mass) {
        CK(cudaMemcpyAsync(c->P.m, mass, n * sizeof(double), cudaMemcpyHostToDevice, st));
      } else {
        ones.assign(n, 1.0);
        CK(cudaMemcpyAsync(c->P.m, ones.data(), n * sizeof(double), cudaMemcpyHostToDevice, st));
      }
      if (vel) {
        CK(cudaMemcpyAsync(c->P.v, vel, 3 * n * sizeof(double), cudaMemcpyHostToDevice, st));
      } else {
        CK(cudaMemsetAsync(c->P.v, 0, 3 * n * sizeof(double), st));
      }
    }
    CK(cudaMemsetAsync(&c->ds->err, 0, sizeof(unsigned int), st));
    CK(cudaMemsetAsync(&c->ds->step, 0, sizeof(long long), st));
    launch_fold_init(m, c->P, pin, nullptr, &c->ds->err, st);
    // Sec. II, Fig. 1: vertex charges, exact Gauss scan into the ledger
    launch_cic(m, c->P, Q, bg, st);
    launch_gauss_scan(m, Q, c->Lg, scr, &c->ds->err, st);
    CKL();
    s = check_err(c);
    if (s == MEMD_OK) {
      // k = 0 mode of D set to -P/V (Sec. V), then relaxation to curl E = 0
      launch_dipole(m, c->P, c->ds, st);
      launch_ledger_sums(m, c->Lg, c->ds, st);
      launch_init_D(m, D64, c->Lg, c->ds, std::ldexp(1.0, -48) / (m.a * m.a), c->Vbox, st);
      CKL();
      // the minimiser through the scalar potential; the relaxation below then
      // only confirms the circulation residual (or, if the potential solve
      // did not converge, relaxes from the scanned field)
      if (c->psi) {
        int its = 0;
        const memd_status ms = mg_relax(c, D64, c->psi, c->eps_eff_inv,
                                        std::min(c->relax_tol, 1e-12), c->relax_maxit, &its);
        if (ms != MEMD_OK) {
          cudaGetLastError();
          launch_init_D(m, D64, c->Lg, c->ds, std::ldexp(1.0, -48) / (m.a * m.a), c->Vbox, st);
        }
      }
      s = relax(c, D64, c->relax_tol, c->relax_maxit);
    }
    if (s == MEMD_OK) {
      c->cur = 0;
      launch_cast(c->prec, c->D(), D64, 3 * m.V, st);
      CK(cudaMemsetAsync(c->B(), 0, 3 * m.V * esz(c), st));
      CK(clear_transfers(c, c->Tb, st));
      if (c->Tb2) CK(cudaMemsetAsync(c->Tb2, 0, kLT * 3 * m.V * sizeof(long long), st));
      c->pending = false;
      CK(cudaMemsetAsync(&c->ds->ticket, 0, sizeof(unsigned int), st));
      const StepParams sp = step_params(c, 0, 0.0, 0.0);
      launch_particle_constants(sp, c->P, st);
      launch_gather(m, c->prec, sp, c->P, c->D(), c->ie, c->ie64, c->ds, 0, 1, st);
      CKL();
      s = check_err(c);
    }
  }
  dfree(c, pin);
  dfree(c, Q);
  dfree(c, scr);
  dfree(c, D64);
  if (s == MEMD_OK) c->initialised = true;
  c->gen += 1;
  return s;
}

// One step on buffer parity `par` (state in buffer par, result in 1 - par).
// The charge transfer of the drift runs on a side stream beside the fused
// field update (neither reads what the other writes; with timing on, after
// it); the transfers are applied to the new D, then the gather closes the
// step.
// a timing event inside a captured graph is an external event node; outside
// capture it is recorded as usual
static cudaError_t record_timing_event(cudaEvent_t ev, cudaStream_t st) {
  cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
  if (cudaStreamIsCapturing(st, &cs) != cudaSuccess) return cudaGetLastError();
  return cs == cudaStreamCaptureStatusActive ? cudaEventRecordWithFlags(ev, st, cudaEventRecordExternal)
                                             : cudaEventRecord(ev, st);
}

static memd_status record_step(memd_ctx* c, const StepParams& sp, int par, bool timed) {
  const Mesh& m = c->mesh;
  const cudaStream_t st = c->stream;
  if (timed) {
    // instrumented: the field update alone between its event pair
    CK(record_timing_event(c->ev0, st));
    launch_field(c, par, sp.coefB, sp.coefD, c->fcfg);
    CK(record_timing_event(c->ev1, st));
    launch_kick_drift_deposit(m, sp, c->P, c->Tb, c->ds, st);
  } else {
    CK(cudaEventRecord(c->fork, st));
    CK(cudaStreamWaitEvent(c->side, c->fork, 0));
    launch_kick_drift_deposit(m, sp, c->P, c->Tb, c->ds, c->side);
    CK(cudaEventRecord(c->join, c->side));
    launch_field(c, par, sp.coefB, sp.coefD, c->fcfg);
    CK(cudaStreamWaitEvent(st, c->join, 0));
  }
  if (apply_dense(c->apply_mode))
    launch_apply_dense(c->prec, 3 * m.V, c->Tb, c->Lg, c->Dbuf[par ^ 1], sp.scale, st);
  else
    launch_apply(m, c->prec, c->P, c->Tb, c->Lg, c->Dbuf[par ^ 1], sp.scale, st);
  launch_gather(m, c->prec, sp, c->P, c->Dbuf[par ^ 1], c->ie, c->ie64, c->ds, 1, 2, st);
  CKL();
  return MEMD_OK;
}

// transfer buffer of buffer parity q of the single-launch step, which leaves
// the transfers of its move, not yet applied, in the buffer of the parity it
// wrote: transfer words only, component major (tw_index with cmV = V), the
// two buffers one after the other in Tb2 (the graph step uses the pairs of
// Tb, and applies them at once)
static long long* tbuf(memd_ctx* c, int q) { return c->Tb2 + q * 3 * c->mesh.V; }

// the whole step as one cooperative launch (same kernels' device functions)
static memd_status record_step_coop(memd_ctx* c, const StepParams& sp, int par, bool timed) {
  const cudaStream_t st = c->stream;
  if (timed) CK(record_timing_event(c->ev0, st));
  const cudaError_t e = launch_step_coop(
      c->mesh, c->prec, sp, c->P, c->Dbuf[par], c->Bbuf[par], c->ie, c->Dbuf[par ^ 1],
      c->Bbuf[par ^ 1], c->ie64, tbuf(c, par), tbuf(c, par ^ 1), c->Lg, c->ds, c->coop_grid,
      coop_zchunk(c->mesh, c->coop_grid), st);
  if (e != cudaSuccess) return fail(c, MEMD_ERR_CUDA, cudaGetErrorString(e));
  if (timed) CK(record_timing_event(c->ev1, st));
  return MEMD_OK;
}

}  // extern "C"

// Apply the transfers a single-launch step left pending (to D and the
// ledger, through the last move's links) before anything reads or replaces
// the state.  (C++ linkage: used by the batch, not part of the C ABI.)
memd_status memd_flush(memd_ctx* c) {
  if (!c->pending) return MEMD_OK;
  launch_apply(c->mesh, c->prec, c->P, tbuf(c, c->cur), c->Lg, c->D(),
               std::ldexp(1.0, -48) / (c->mesh.a * c->mesh.a), c->stream, c->mesh.V);
  c->pending = false;
  if (cudaGetLastError() != cudaSuccess) return fail(c, MEMD_ERR_CUDA, "applying pending transfers");
  return MEMD_OK;
}

extern "C" {

// single launch or graph of four kernels for this system (decided when the
// step graphs are built, once the particle count is known)
static bool want_coop(const memd_ctx* c) {
  if (c->coop_grid <= 0 || c->step_engine == MEMD_STEP_GRAPH) return false;
  if (c->step_engine == MEMD_STEP_SINGLE) return true;
  return c->mesh.V <= (int64_t(1) << 17) && c->P.n <= (int64_t)16 * c->coop_grid;
}

// Errors raised by kernels of earlier batches, without blocking: the flag is
// copied back after each batch and read once that copy has completed.
static memd_status poll_err(memd_ctx* c, bool block) {
  if (block) return check_err(c);
  return MEMD_OK;
}

// what every step needs before it is launched: the per-particle constants
// of this thermostat, the engine (decided when the step graphs are built),
// the second transfer buffer of the single launch, applied transfers for the
// graph engine, the tuned field kernel
static memd_status step_prepare(memd_ctx* c, const memd_thermostat* th, StepParams& sp) {
  const int thermo = th ? 1 : 0;
  const double gamma = th ? th->gamma : 0.0, kT = th ? th->kT : 0.0;
  sp = step_params(c, thermo, gamma, kT);
  if (c->graph_thermo != thermo || c->graph_gamma != gamma || c->graph_kT != kT || !c->sig_ready) {
    drop_graphs(c);
    // per-particle Langevin amplitude for this thermostat (same expression as per step)
    launch_particle_constants(sp, c->P, c->stream);
    c->sig_ready = true;
    c->graph_thermo = thermo;
    c->graph_gamma = gamma;
    c->graph_kT = kT;
  }
  if (!c->graph[0] && !c->graph[1]) c->coop = want_coop(c);
  if (c->coop && !c->Tb2) {
    // the single-launch step's two transfer buffers (3 V words each)
    c->Tb2 = (long long*)dalloc(c, kLT * 3 * c->mesh.V * sizeof(long long));
    if (!c->Tb2) return fail(c, MEMD_ERR_OOM, "second transfer buffer");
    CK(cudaMemsetAsync(c->Tb2, 0, kLT * 3 * c->mesh.V * sizeof(long long), c->stream));
  }
  if (!c->coop) {
    const memd_status e = memd_flush(c);
    if (e != MEMD_OK) return e;
  }
  if (!c->coop && !c->fcfg_ready) {
    const memd_status e = autotune_fused(c);
    if (e != MEMD_OK) return e;
    c->fcfg_ready = true;
  }
  return MEMD_OK;
}

memd_status memd_step(memd_ctx* c, int64_t nsteps, const memd_thermostat* th) {
  memd::NvtxRange nvtx_("memd_step");
  if (!c) return MEMD_ERR_INVALID;
  if (!c->initialised) return fail(c, MEMD_ERR_STATE, "memd_init_field first");
  if (nsteps < 0) return fail(c, MEMD_ERR_INVALID, "negative step count");
  CK(cudaSetDevice(c->device));
  const int thermo = th ? 1 : 0;
  const double gamma = th ? th->gamma : 0.0, kT = th ? th->kT : 0.0;
  StepParams sp;
  {
    const memd_status e = step_prepare(c, th, sp);
    if (e != MEMD_OK) return e;
  }
  const bool timed = c->time_kernels != 0;
  auto record = [&](int par) {
    return c->coop ? record_step_coop(c, sp, par, timed) : record_step(c, sp, par, timed);
  };
  for (int64_t s = 0; s < nsteps; ++s) {
    const int par = c->cur;
    harvest_timing(c);
    if (!c->use_graphs || (c->coop && !c->coop_graph_ok)) {
      memd_status r = record(par);
      if (r != MEMD_OK) return r;
    } else {
      if (!c->graph[par]) {
        cudaGraph_t g = nullptr;
        CK(cudaStreamBeginCapture(c->stream, cudaStreamCaptureModeThreadLocal));
        memd_status r = record(par);
        cudaError_t e = cudaStreamEndCapture(c->stream, &g);
        cudaError_t ie = cudaErrorUnknown;
        if (r == MEMD_OK && e == cudaSuccess) ie = cudaGraphInstantiate(&c->graph[par], g, 0);
        if (g) cudaGraphDestroy(g);
        if (ie != cudaSuccess && c->coop) {
          // a cooperative launch that cannot be captured or replayed: launch
          // it directly from now on
          cudaGetLastError();
          c->graph[par] = nullptr;
          c->coop_graph_ok = false;
          memd_status r2 = record(par);
          if (r2 != MEMD_OK) return r2;
          c->timing_pending = timed;
          c->cur = par ^ 1;
          c->pending = true;
          continue;
        }
        if (r != MEMD_OK) return r;
        if (e != cudaSuccess) return fail(c, MEMD_ERR_CUDA, "graph capture");
        if (ie != cudaSuccess) return fail(c, MEMD_ERR_CUDA, "graph instantiate");
        c->graph_thermo = thermo;
        c->graph_gamma = gamma;
        c->graph_kT = kT;
      }
      CK(cudaGraphLaunch(c->graph[par], c->stream));
    }
    c->timing_pending = timed;
    c->cur = par ^ 1;
    if (c->coop) c->pending = true;
  }
  return poll_err(c, false);
}

memd_status memd_forces(memd_ctx* c, double* f_out) {
  if (!c || !f_out) return MEMD_ERR_INVALID;
  if (!c->initialised) return fail(c, MEMD_ERR_STATE, "memd_init_field first");
  CK(cudaSetDevice(c->device));
  if (c->P.n > 0)
    CK(cudaMemcpyAsync(f_out, c->P.F, 3 * c->P.n * sizeof(double), cudaMemcpyDeviceToHost,
                       c->stream));
  return check_err(c);
}

memd_status memd_forces_device(memd_ctx* c, const double** f_dev) {
  if (!c || !f_dev) return MEMD_ERR_INVALID;
  if (!c->initialised) return fail(c, MEMD_ERR_STATE, "memd_init_field first");
  *f_dev = c->P.F;
  return MEMD_OK;
}

memd_status memd_energy(memd_ctx* c, memd_energy_terms* out) {
  if (!c || !out) return MEMD_ERR_INVALID;
  if (!c->initialised) return fail(c, MEMD_ERR_STATE, "memd_init_field first");
  CK(cudaSetDevice(c->device));
  {
    const memd_status fe = memd_flush(c);
    if (fe != MEMD_OK) return fe;
  }
  const Mesh& m = c->mesh;
  const cudaStream_t st = c->stream;
  const int R = reduce_blocks();
  double* part = c->red;
  double* sc = scal(c);
  const StepParams sp = step_params(c, 0, 0, 0);
  launch_field_energy(m, c->prec, c->D(), c->B(), c->ie, sp.coefB, part, part + R, st);
  launch_finish(part, 0, sc + 8, st);
  launch_finish(part + R, 0, sc + 9, st);
  launch_particle_energy(m, sp, c->P, c->ie64, part + 2 * R, part + 3 * R, st);
  launch_finish(part + 2 * R, 0, sc + 10, st);
  launch_finish(part + 3 * R, 0, sc + 11, st);
  long long qtot = 0;
  long long* Q = (long long*)dalloc(c, sizeof(long long) * m.V + 64);
  if (!Q) return fail(c, MEMD_ERR_OOM, "energy scratch");
  unsigned long long* mism = (unsigned long long*)(Q + m.V);
  // background of a non-neutral system, from the valences on the device
  std::vector<int> hq(c->P.n > 0 ? c->P.n : 1);
  if (c->P.n > 0)
    CK(cudaMemcpyAsync(hq.data(), c->P.q, c->P.n * sizeof(int), cudaMemcpyDeviceToHost, st));
  CK(cudaStreamSynchronize(st));
  for (int64_t p = 0; p < c->P.n; ++p) qtot += hq[p];
  const long long bg = (long long)(((__int128)qtot << 48) / m.V);
  launch_cic(m, c->P, Q, bg, st);
  CK(cudaMemsetAsync(mism, 0, sizeof(unsigned long long), st));
  launch_gauss_check(m, c->prec, c->D(), c->Lg, Q, m.a * m.a, part, mism, st);
  launch_finish(part, 1, sc + 12, st);
  CKL();
  double h[5];
  unsigned long long bad = 0;
  long long Pl[3], step = 0;
  CK(cudaMemcpyAsync(h, sc + 8, 5 * sizeof(double), cudaMemcpyDeviceToHost, st));
  CK(cudaMemcpyAsync(&bad, mism, sizeof(bad), cudaMemcpyDeviceToHost, st));
  CK(cudaMemcpyAsync(Pl, c->ds->Plast, sizeof(Pl), cudaMemcpyDeviceToHost, st));
  CK(cudaMemcpyAsync(&step, &c->ds->step, sizeof(step), cudaMemcpyDeviceToHost, st));
  CK(cudaStreamSynchronize(st));
  dfree(c, Q);
  const double a3 = m.a * m.a * m.a;
  out->electric = h[0] * a3;
  out->magnetic = h[1] * 0.5 * c->c * c->c * a3;
  out->kinetic = h[2];
  out->self = c->self_mode ? h[3] : 0.0;
  for (int d = 0; d < 3; ++d) out->P[d] = (double)Pl[d] * (m.a / (double)kS);
  double dip = 0.0;
  if (c->dipole_corr)
    for (int e = 0; e < 3; ++e)
      for (int d = 0; d < 3; ++d) dip += 0.5 * out->P[e] * c->Minv[3 * e + d] * out->P[d] / c->Vbox;
  out->dipole = dip;
  out->total = out->kinetic + out->electric + out->magnetic - out->self - out->dipole;
  out->gauss_residual = h[4];
  out->gauss_exact = bad == 0 ? 1 : 0;
  out->pad = 0;
  out->step = step;
  return check_err(c);
}

memd_status memd_dipole_check(memd_ctx* c, double limit, double* ratio) {
  if (!c || !(limit > 0.0)) return MEMD_ERR_INVALID;
  if (!c->initialised) return fail(c, MEMD_ERR_STATE, "memd_init_field first");
  CK(cudaSetDevice(c->device));
  {
    const memd_status fe = memd_flush(c);
    if (fe != MEMD_OK) return fe;
  }
  const Mesh& m = c->mesh;
  const cudaStream_t st = c->stream;
  double* part = c->red;
  double* sc = scal(c);
  const int R = reduce_blocks();
  launch_field_moments(c->prec, c->D(), c->ie, m.V, part, st);
  for (int k = 0; k < 4; ++k) launch_finish(part + k * R, 0, sc + 8 + k, st);
  CKL();
  double h[4];
  long long Pl[3];
  CK(cudaMemcpyAsync(h, sc + 8, 4 * sizeof(double), cudaMemcpyDeviceToHost, st));
  CK(cudaMemcpyAsync(Pl, c->ds->Plast, sizeof(Pl), cudaMemcpyDeviceToHost, st));
  CK(cudaStreamSynchronize(st));
  // the correction's field eps_eff^-1 P / V, as the gather applies it
  double P[3], E[3], mp2 = 0.0;
  for (int d = 0; d < 3; ++d) P[d] = (double)Pl[d] * (m.a / (double)kS);
  for (int e = 0; e < 3; ++e) {
    E[e] = (c->Minv[3 * e] * P[0] + c->Minv[3 * e + 1] * P[1] + c->Minv[3 * e + 2] * P[2]) / c->Vbox;
    mp2 += E[e] * E[e];
  }
  // the field of the charges about its mean: sum_d mean over the d-links of
  // (E_d - mean E_d)^2 = sum_d mean(E_d^2) - sum_d (mean E_d)^2
  const double Vd = (double)m.V;
  double fl2 = h[0] / Vd;
  for (int d = 0; d < 3; ++d) fl2 -= (h[1 + d] / Vd) * (h[1 + d] / Vd);
  const double efl = std::sqrt(std::max(fl2, 0.0));
  const double r = efl > 0.0 ? std::sqrt(mp2) / efl : (mp2 > 0.0 ? HUGE_VAL : 0.0);
  if (ratio) *ratio = r;
  const memd_status s = check_err(c);
  if (s != MEMD_OK) return s;
  if (r > limit)
    return fail(c, MEMD_ERR_DIPOLE_DRIFT,
                "the dipole correction outgrew the lattice field: re-initialise the field");
  return MEMD_OK;
}

memd_status memd_inject(memd_ctx* c, int32_t kind, double wait_s) {
  if (!c) return MEMD_ERR_INVALID;
  if (kind != MEMD_INJECT_NONE && kind != MEMD_INJECT_BARRIER_SKEW)
    return fail(c, MEMD_ERR_INVALID, "unknown injection");
  if (!(wait_s >= 0.0) || wait_s > 10.0) return fail(c, MEMD_ERR_INVALID, "wait bound out of range");
  CK(cudaSetDevice(c->device));
  drop_graphs(c);  // the step graphs hold the wait bound
  c->wait_ns = wait_s > 0.0 ? (unsigned long long)(wait_s * 1e9) : kBarrierWaitNs;
  if (kind == MEMD_INJECT_BARRIER_SKEW) {
    if (!c->initialised) return fail(c, MEMD_ERR_STATE, "memd_init_field first");
    if (!c->coop) return fail(c, MEMD_ERR_STATE, "the steps of this context have no grid barrier");
    // one extra arrival: the next barrier's count cannot reach its target
    unsigned long long n = 0;
    CK(cudaStreamSynchronize(c->stream));
    CK(cudaMemcpy(&n, &c->ds->bar_arrivals, sizeof(n), cudaMemcpyDeviceToHost));
    n += 1;
    CK(cudaMemcpy(&c->ds->bar_arrivals, &n, sizeof(n), cudaMemcpyHostToDevice));
  }
  return MEMD_OK;
}

memd_status memd_get_particles(memd_ctx* c, double* pos, double* vel, int32_t* img) {
  if (!c) return MEMD_ERR_INVALID;
  if (!c->initialised) return fail(c, MEMD_ERR_STATE, "memd_init_field first");
  CK(cudaSetDevice(c->device));
  const size_t n = (size_t)c->P.n;
  if (n) {
    if (pos) CK(cudaMemcpyAsync(pos, c->P.x, 3 * n * sizeof(double), cudaMemcpyDeviceToHost, c->stream));
    if (vel) CK(cudaMemcpyAsync(vel, c->P.v, 3 * n * sizeof(double), cudaMemcpyDeviceToHost, c->stream));
    if (img) CK(cudaMemcpyAsync(img, c->P.img, 3 * n * sizeof(int), cudaMemcpyDeviceToHost, c->stream));
  }
  return check_err(c);
}

// state load on the stream (no synchronisation): velocities, positions with
// their image counters folded on the device, or image counters alone.  The
// transfers a single-launch step left pending concern D and the ledger
// only, so the load itself does not need them applied.
static memd_status load_particles(memd_ctx* c, const double* pos, const double* vel,
                                  const int32_t* img, bool flush) {
  if (flush) {
    const memd_status fe = memd_flush(c);
    if (fe != MEMD_OK) return fe;
  }
  const size_t n = (size_t)c->P.n;
  if (!n) return MEMD_OK;
  const cudaStream_t st = c->stream;
  if (vel) CK(cudaMemcpyAsync(c->P.v, vel, 3 * n * sizeof(double), cudaMemcpyHostToDevice, st));
  if (pos) {
    double* pin = c->pin;
    int* iin = (int*)(pin + 3 * n);
    CK(cudaMemcpyAsync(pin, pos, 3 * n * sizeof(double), cudaMemcpyHostToDevice, st));
    if (img)
      CK(cudaMemcpyAsync(iin, img, 3 * n * sizeof(int), cudaMemcpyHostToDevice, st));
    else
      CK(cudaMemcpyAsync(iin, c->P.img, 3 * n * sizeof(int), cudaMemcpyDeviceToDevice, st));
    launch_fold_init(c->mesh, c->P, pin, iin, &c->ds->err, st);
    CKL();
  } else if (img) {
    CK(cudaMemcpyAsync(c->P.img, img, 3 * n * sizeof(int), cudaMemcpyHostToDevice, st));
  }
  return MEMD_OK;
}

memd_status memd_set_particles(memd_ctx* c, const double* pos, const double* vel,
                               const int32_t* img) {
  if (!c) return MEMD_ERR_INVALID;
  if (!c->initialised) return fail(c, MEMD_ERR_STATE, "memd_init_field first");
  CK(cudaSetDevice(c->device));
  const memd_status s = load_particles(c, pos, vel, img, true);
  if (s != MEMD_OK) return s;
  return check_err(c);  // synchronises the stream
}

memd_status memd_step_host(memd_ctx* c, const double* pos_in, const double* vel_in,
                           const int32_t* img_in, int64_t nsteps, const memd_thermostat* th,
                           double* pos_out, double* vel_out, int32_t* img_out, double* f_out) {
  if (!c) return MEMD_ERR_INVALID;
  if (!c->initialised) return fail(c, MEMD_ERR_STATE, "memd_init_field first");
  if (nsteps < 0) return fail(c, MEMD_ERR_INVALID, "negative step count");
  CK(cudaSetDevice(c->device));
  if (!c->err_host) {
    if (cudaHostAlloc((void**)&c->err_host, sizeof(unsigned int), cudaHostAllocDefault) !=
        cudaSuccess) {
      cudaGetLastError();
      c->err_host = nullptr;
      return fail(c, MEMD_ERR_OOM, "pinned error word");
    }
  }
  memd_status s = MEMD_OK;
  if (pos_in || vel_in || img_in) {
    s = load_particles(c, pos_in, vel_in, img_in, false);
    if (s != MEMD_OK) return s;
  }
  s = memd_step(c, nsteps, th);
  if (s != MEMD_OK) return s;
  const size_t n = (size_t)c->P.n;
  const cudaStream_t st = c->stream;
  if (n) {
    if (pos_out) CK(cudaMemcpyAsync(pos_out, c->P.x, 3 * n * sizeof(double), cudaMemcpyDeviceToHost, st));
    if (vel_out) CK(cudaMemcpyAsync(vel_out, c->P.v, 3 * n * sizeof(double), cudaMemcpyDeviceToHost, st));
    if (img_out) CK(cudaMemcpyAsync(img_out, c->P.img, 3 * n * sizeof(int), cudaMemcpyDeviceToHost, st));
    if (f_out) CK(cudaMemcpyAsync(f_out, c->P.F, 3 * n * sizeof(double), cudaMemcpyDeviceToHost, st));
  }
  CK(cudaMemcpyAsync(c->err_host, &c->ds->err, sizeof(unsigned int), cudaMemcpyDeviceToHost, st));
  CK(cudaStreamSynchronize(st));
  if (*c->err_host) return check_err(c);
  return MEMD_OK;
}

// the I/O block for the present particle count (page-locked host copy and
// its device mirror), allocated on first use and after a particle count change
static memd_status io_block(memd_ctx* c) {
  if (c->io_n == c->P.n && c->io_host && c->io_dev) return MEMD_OK;
  drop_graphs(c);  // the round-trip graphs hold the old block's addresses
  if (c->io_host) cudaFreeHost(c->io_host);
  dfree(c, c->io_dev);
  c->io_host = nullptr;
  c->io_dev = nullptr;
  c->io_n = -1;
  const IoLayout L = io_layout(c->P.n);
  if (cudaHostAlloc((void**)&c->io_host, (size_t)L.bytes, cudaHostAllocDefault) != cudaSuccess) {
    cudaGetLastError();
    c->io_host = nullptr;
    return fail(c, MEMD_ERR_OOM, "page-locked I/O block");
  }
  std::memset(c->io_host, 0, (size_t)L.bytes);
  c->io_dev = dalloc(c, (size_t)L.bytes);
  if (!c->io_dev) return fail(c, MEMD_ERR_OOM, "device I/O block");
  c->io_n = c->P.n;
  return MEMD_OK;
}

memd_status memd_io_buffers(memd_ctx* c, memd_io* io) {
  if (!c || !io) return MEMD_ERR_INVALID;
  if (!c->initialised) return fail(c, MEMD_ERR_STATE, "memd_init_field first");
  CK(cudaSetDevice(c->device));
  const memd_status s = io_block(c);
  if (s != MEMD_OK) return s;
  const IoLayout L = io_layout(c->P.n);
  io->pos = (double*)(c->io_host + L.pos);
  io->vel = (double*)(c->io_host + L.vel);
  io->img = (int32_t*)(c->io_host + L.img);
  io->f = (double*)(c->io_host + L.f);
  return MEMD_OK;
}

memd_status memd_step_io(memd_ctx* c, int32_t load, int64_t nsteps, const memd_thermostat* th) {
  memd::NvtxRange nvtx_("memd_step_io");
  if (!c) return MEMD_ERR_INVALID;
  if (!c->initialised) return fail(c, MEMD_ERR_STATE, "memd_init_field first");
  if (nsteps < 0) return fail(c, MEMD_ERR_INVALID, "negative step count");
  CK(cudaSetDevice(c->device));
  memd_status s = io_block(c);
  if (s != MEMD_OK) return s;
  const IoLayout L = io_layout(c->P.n);
  const cudaStream_t st = c->stream;
  if (load && nsteps == 1 && c->P.n > 0 && c->use_graphs && c->io_graph_ok) {
    // the usual host loop: one graph launch a call
    StepParams sp;
    s = step_prepare(c, th, sp);
    if (s != MEMD_OK) return s;
    if (!c->coop || c->coop_graph_ok) {
      const bool timed = c->time_kernels != 0;
      const int par = c->cur;
      harvest_timing(c);
      if (!c->io_graph[par]) {
        cudaGraph_t g = nullptr;
        CK(cudaStreamBeginCapture(st, cudaStreamCaptureModeThreadLocal));
        cudaMemcpyAsync(c->io_dev, c->io_host, (size_t)L.f, cudaMemcpyHostToDevice, st);
        launch_io_unpack(c->mesh, c->P, c->io_dev, &c->ds->err, st);
        const memd_status r = c->coop ? record_step_coop(c, sp, par, timed)
                                      : record_step(c, sp, par, timed);
        launch_io_pack(c->P, c->io_dev, &c->ds->err, st);
        cudaMemcpyAsync(c->io_host, c->io_dev, (size_t)L.bytes, cudaMemcpyDeviceToHost, st);
        const cudaError_t e = cudaStreamEndCapture(st, &g);
        cudaError_t ie = cudaErrorUnknown;
        if (r == MEMD_OK && e == cudaSuccess) ie = cudaGraphInstantiate(&c->io_graph[par], g, 0);
        if (g) cudaGraphDestroy(g);
        if (ie != cudaSuccess) {  // not capturable here: copies and step one by one
          cudaGetLastError();
          c->io_graph[par] = nullptr;
          c->io_graph_ok = false;
        }
      }
      if (c->io_graph[par]) {
        CK(cudaGraphLaunch(c->io_graph[par], st));
        c->timing_pending = timed;
        c->cur = par ^ 1;
        if (c->coop) c->pending = true;
        CK(cudaStreamSynchronize(st));
        if (*(const unsigned int*)(c->io_host + L.err)) return check_err(c);
        return MEMD_OK;
      }
    }
  }
  if (load && c->P.n > 0) {
    // positions, velocities and image counters: the first 60 n bytes
    CK(cudaMemcpyAsync(c->io_dev, c->io_host, (size_t)L.f, cudaMemcpyHostToDevice, st));
    launch_io_unpack(c->mesh, c->P, c->io_dev, &c->ds->err, st);
    CKL();
  }
  s = memd_step(c, nsteps, th);
  if (s != MEMD_OK) return s;
  launch_io_pack(c->P, c->io_dev, &c->ds->err, st);
  CKL();
  CK(cudaMemcpyAsync(c->io_host, c->io_dev, (size_t)L.bytes, cudaMemcpyDeviceToHost, st));
  CK(cudaStreamSynchronize(st));
  if (*(const unsigned int*)(c->io_host + L.err)) return check_err(c);
  return MEMD_OK;
}

memd_status memd_move(memd_ctx* c, const double* pos, const int32_t* img) {
  if (!c || !pos) return MEMD_ERR_INVALID;
  if (!c->initialised) return fail(c, MEMD_ERR_STATE, "memd_init_field first");
  CK(cudaSetDevice(c->device));
  {
    const memd_status fe = memd_flush(c);
    if (fe != MEMD_OK) return fe;
  }
  const size_t n = (size_t)c->P.n;
  if (!n) return MEMD_OK;
  const cudaStream_t st = c->stream;
  double* pin = c->pin;
  int* iin = (int*)(pin + 3 * n);
  CK(cudaMemcpyAsync(pin, pos, 3 * n * sizeof(double), cudaMemcpyHostToDevice, st));
  if (img) CK(cudaMemcpyAsync(iin, img, 3 * n * sizeof(int), cudaMemcpyHostToDevice, st));
  CK(cudaMemsetAsync(c->ds->Pacc, 0, sizeof(c->ds->Pacc), st));
  launch_move_deposit(c->mesh, c->P, pin, img ? iin : nullptr, c->Tb, c->ds, st);
  launch_apply(c->mesh, c->prec, c->P, c->Tb, c->Lg, c->D(),
               std::ldexp(1.0, -48) / (c->mesh.a * c->mesh.a), st);
  launch_step_end(c->ds, 0, st);
  CKL();
  return check_err(c);
}

memd_status memd_get_fields(memd_ctx* c, double* D, double* B, int64_t* Lg) {
  if (!c) return MEMD_ERR_INVALID;
  CK(cudaSetDevice(c->device));
  {
    const memd_status fe = memd_flush(c);
    if (fe != MEMD_OK) return fe;
  }
  const size_t n3 = 3 * (size_t)c->mesh.V;
  const cudaStream_t st = c->stream;
  double* tmp = (double*)dalloc(c, n3 * sizeof(double));
  if (!tmp) return fail(c, MEMD_ERR_OOM, "get_fields scratch");
  if (D) {
    launch_widen(c->prec, tmp, c->D(), (int64_t)n3, st);
    CK(cudaMemcpyAsync(D, tmp, n3 * sizeof(double), cudaMemcpyDeviceToHost, st));
    CK(cudaStreamSynchronize(st));
  }
  if (B) {
    launch_widen(c->prec, tmp, c->B(), (int64_t)n3, st);
    CK(cudaMemcpyAsync(B, tmp, n3 * sizeof(double), cudaMemcpyDeviceToHost, st));
    CK(cudaStreamSynchronize(st));
  }
  if (Lg) CK(ledger_to_host(c, Lg, st));
  CK(cudaStreamSynchronize(st));
  dfree(c, tmp);
  return MEMD_OK;
}

memd_status memd_set_fields(memd_ctx* c, const double* D, const double* B, const int64_t* Lg) {
  if (!c) return MEMD_ERR_INVALID;
  CK(cudaSetDevice(c->device));
  {
    const memd_status fe = memd_flush(c);
    if (fe != MEMD_OK) return fe;
  }
  const size_t n3 = 3 * (size_t)c->mesh.V;
  const cudaStream_t st = c->stream;
  double* tmp = (double*)dalloc(c, n3 * sizeof(double));
  if (!tmp) return fail(c, MEMD_ERR_OOM, "set_fields scratch");
  if (D) {
    CK(cudaMemcpyAsync(tmp, D, n3 * sizeof(double), cudaMemcpyHostToDevice, st));
    launch_cast(c->prec, c->D(), tmp, (int64_t)n3, st);
    CK(cudaStreamSynchronize(st));
  }
  if (B) {
    CK(cudaMemcpyAsync(tmp, B, n3 * sizeof(double), cudaMemcpyHostToDevice, st));
    launch_cast(c->prec, c->B(), tmp, (int64_t)n3, st);
    CK(cudaStreamSynchronize(st));
  }
  if (Lg) CK(ledger_from_host(c, Lg, st));
  CKL();
  CK(cudaStreamSynchronize(st));
  dfree(c, tmp);
  return MEMD_OK;
}

// ----------------------------------------------------- checkpoint / resume
// A saved state: this header, then D and B in the field precision, the
// ledger, and the particle arrays x, v, F, Ft (FP64), img, q (int32), m.
struct StateHeader {
  char magic[8];
  int32_t version, prec;
  int32_t mesh[3], pad;
  int64_t n, step;
  int64_t Plast[3];
  double box[3];
};
static const char kStateMagic[8] = {'M', 'E', 'M', 'D', 'S', 'T', 'A', 'T'};

int64_t memd_state_bytes(const memd_ctx* c) {
  if (!c) return 0;
  const int64_t V3 = 3 * c->mesh.V, n = c->P.n;
  return (int64_t)sizeof(StateHeader) + V3 * (2 * (int64_t)memd_esz(c) + 8) + n * 120;
}

memd_status memd_save_state(memd_ctx* c, void* buf, int64_t bytes) {
  if (!c || !buf) return MEMD_ERR_INVALID;
  if (!c->initialised) return fail(c, MEMD_ERR_STATE, "memd_init_field first");
  if (bytes < memd_state_bytes(c)) return fail(c, MEMD_ERR_INVALID, "state buffer too small");
  CK(cudaSetDevice(c->device));
  {
    const memd_status fe = memd_flush(c);
    if (fe != MEMD_OK) return fe;
  }
  const cudaStream_t st = c->stream;
  const size_t V3 = 3 * (size_t)c->mesh.V, n = (size_t)c->P.n, es = memd_esz(c);
  StateHeader h;
  std::memset(&h, 0, sizeof(h));
  std::memcpy(h.magic, kStateMagic, 8);
  h.version = 1;
  h.prec = c->prec;
  for (int d = 0; d < 3; ++d) {
    h.mesh[d] = c->mesh.n[d];
    h.box[d] = c->mesh.L[d];
  }
  h.n = (int64_t)n;
  CK(cudaMemcpyAsync(&h.step, &c->ds->step, sizeof(long long), cudaMemcpyDeviceToHost, st));
  CK(cudaMemcpyAsync(h.Plast, c->ds->Plast, 3 * sizeof(long long), cudaMemcpyDeviceToHost, st));
  char* p = (char*)buf + sizeof(StateHeader);
  bool ok = true;
  auto get = [&](const void* src, size_t b) {
    if (b && cudaMemcpyAsync(p, src, b, cudaMemcpyDeviceToHost, st) != cudaSuccess) ok = false;
    p += b;
  };
  get(c->D(), V3 * es);
  get(c->B(), V3 * es);
  if (ok && ledger_to_host(c, p, st) != cudaSuccess) ok = false;
  p += V3 * 8;
  get(c->P.x, 3 * n * 8);
  get(c->P.v, 3 * n * 8);
  get(c->P.F, 3 * n * 8);
  get(c->P.Ft, 3 * n * 8);
  get(c->P.img, 3 * n * 4);
  get(c->P.q, n * 4);
  get(c->P.m, n * 8);
  if (!ok) return fail(c, MEMD_ERR_CUDA, "state copy");
  CK(cudaStreamSynchronize(st));
  std::memcpy(buf, &h, sizeof(h));
  return check_err(c);
}

memd_status memd_load_state(memd_ctx* c, const void* buf, int64_t bytes) {
  if (!c || !buf) return MEMD_ERR_INVALID;
  if (!c->initialised) return fail(c, MEMD_ERR_STATE, "memd_init_field first");
  StateHeader h;
  if (bytes < (int64_t)sizeof(h)) return fail(c, MEMD_ERR_INVALID, "state buffer too small");
  std::memcpy(&h, buf, sizeof(h));
  if (std::memcmp(h.magic, kStateMagic, 8) != 0 || h.version != 1)
    return fail(c, MEMD_ERR_INVALID, "not a saved state");
  if (h.prec != c->prec || h.n != c->P.n || h.mesh[0] != c->mesh.n[0] ||
      h.mesh[1] != c->mesh.n[1] || h.mesh[2] != c->mesh.n[2] || h.box[0] != c->mesh.L[0] ||
      h.box[1] != c->mesh.L[1] || h.box[2] != c->mesh.L[2])
    return fail(c, MEMD_ERR_INVALID, "saved state of another mesh, precision or particle count");
  if (bytes < memd_state_bytes(c)) return fail(c, MEMD_ERR_INVALID, "state buffer too small");
  {
    // the particle arrays are checked before anything is copied: a saved
    // state holds folded positions (the deposition indexes cells by them),
    // valences in range and positive masses
    const size_t V3 = 3 * (size_t)c->mesh.V, n = (size_t)c->P.n;
    const char* base = (const char*)buf + sizeof(StateHeader) + V3 * (2 * memd_esz(c) + 8);
    // x, v, F, Ft (3n doubles each), img (3n int32), q (n int32), m (n doubles)
    const char* x = base;
    const char* q = base + 3 * n * 8 * 4 + 3 * n * 4;
    const char* ms = q + n * 4;
    for (size_t i = 0; i < n; ++i) {
      double xi[3], mi;
      int32_t qi;
      std::memcpy(xi, x + 24 * i, sizeof(xi));  // the caller's buffer may be unaligned
      std::memcpy(&qi, q + 4 * i, sizeof(qi));
      std::memcpy(&mi, ms + 8 * i, sizeof(mi));
      for (int d = 0; d < 3; ++d)
        if (!(xi[d] >= 0.0 && xi[d] < c->mesh.L[d]))
          return fail(c, MEMD_ERR_INVALID, "saved position outside the box");
      if (qi > 32767 || qi < -32767) return fail(c, MEMD_ERR_INVALID, "saved valence out of range");
      if (!(mi > 0.0) || !std::isfinite(mi))
        return fail(c, MEMD_ERR_INVALID, "saved mass not positive and finite");
    }
  }
  CK(cudaSetDevice(c->device));
  const cudaStream_t st = c->stream;
  drop_graphs(c);
  harvest_timing(c);
  CK(cudaStreamSynchronize(st));
  const size_t V3 = 3 * (size_t)c->mesh.V, n = (size_t)c->P.n, es = memd_esz(c);
  const char* p = (const char*)buf + sizeof(StateHeader);
  bool ok = true;
  auto put = [&](void* dst, size_t b) {
    if (b && cudaMemcpyAsync(dst, p, b, cudaMemcpyHostToDevice, st) != cudaSuccess) ok = false;
    p += b;
  };
  put(c->D(), V3 * es);
  put(c->B(), V3 * es);
  if (ok && ledger_from_host(c, p, st) != cudaSuccess) ok = false;
  p += V3 * 8;
  put(c->P.x, 3 * n * 8);
  put(c->P.v, 3 * n * 8);
  put(c->P.F, 3 * n * 8);
  put(c->P.Ft, 3 * n * 8);
  put(c->P.img, 3 * n * 4);
  put(c->P.q, n * 4);
  put(c->P.m, n * 8);
  if (!ok) return fail(c, MEMD_ERR_CUDA, "state copy");
  // transfers none pending, the step counter and last dipole of the saved
  // state, the accumulators clear; the per-particle constants are formed
  // again from the masses at the next step
  CK(clear_transfers(c, c->Tb, st));
  if (c->Tb2) CK(cudaMemsetAsync(c->Tb2, 0, kLT * 3 * c->mesh.V * sizeof(long long), st));
  c->pending = false;
  CK(cudaMemcpyAsync(&c->ds->step, &h.step, sizeof(long long), cudaMemcpyHostToDevice, st));
  CK(cudaMemcpyAsync(c->ds->Plast, h.Plast, 3 * sizeof(long long), cudaMemcpyHostToDevice, st));
  CK(cudaMemsetAsync(c->ds->Pacc, 0, sizeof(c->ds->Pacc), st));
  CK(cudaMemsetAsync(&c->ds->ticket, 0, sizeof(unsigned int), st));
  CK(cudaStreamSynchronize(st));
  c->sig_ready = false;
  c->gen += 1;
  return check_err(c);
}

memd_status memd_compute_forces(memd_ctx* c) {
  if (!c) return MEMD_ERR_INVALID;
  if (!c->initialised) return fail(c, MEMD_ERR_STATE, "memd_init_field first");
  CK(cudaSetDevice(c->device));
  {
    const memd_status fe = memd_flush(c);
    if (fe != MEMD_OK) return fe;
  }
  const cudaStream_t st = c->stream;
  const StepParams sp = step_params(c, 0, 0.0, 0.0);
  launch_dipole(c->mesh, c->P, c->ds, st);
  launch_gather(c->mesh, c->prec, sp, c->P, c->D(), c->ie, c->ie64, c->ds, 0, 1, st);
  CKL();
  return check_err(c);
}

// A new permittivity on a live context (moving or re-shaped dielectric
// backgrounds).  Gauss' law constrains D, not E, so the present D stays
// valid; with relax_field it is rebuilt from the exact ledger and relaxed to
// the electrostatic minimum of the new medium, as memd_init_field does.
static memd_status set_eps_impl(memd_ctx* c, const memd_eps_profile* eps, int32_t relax_field,
                                const double* dev_values);

memd_status memd_set_eps(memd_ctx* c, const memd_eps_profile* eps, int32_t relax_field) {
  memd::NvtxRange nvtx_("memd_set_eps");
  if (!c) return MEMD_ERR_INVALID;
  if (!eps) return fail(c, MEMD_ERR_INVALID, "no permittivity profile");
  if (!eps_valid(eps, c->mesh.L, c->mesh.a)) return fail(c, MEMD_ERR_INVALID, "permittivity profile");
  CK(cudaSetDevice(c->device));
  return set_eps_impl(c, eps, relax_field, nullptr);
}

memd_status memd_eps_from_density(memd_ctx* c, const memd_salt_rule* rule, int32_t relax_field,
                                  double* eps_out) {
  memd::NvtxRange nvtx_("memd_eps_from_density");
  if (!c || !rule) return MEMD_ERR_INVALID;
  const double r4[4] = {rule->eps0, rule->slope, rule->eps_lo, rule->eps_hi};
  for (double v : r4)
    if (!std::isfinite(v)) return fail(c, MEMD_ERR_INVALID, "salt rule not finite");
  if (!(rule->eps_lo > 0.0) || rule->eps_hi < rule->eps_lo || !(rule->sigma >= 0.0) ||
      rule->sigma > 64.0)
    return fail(c, MEMD_ERR_INVALID, "salt rule out of range");
  if (!c->initialised) return fail(c, MEMD_ERR_STATE, "memd_init_field first");
  CK(cudaSetDevice(c->device));
  {
    const memd_status fe = memd_flush(c);
    if (fe != MEMD_OK) return fe;
  }
  const Mesh& m = c->mesh;
  const cudaStream_t st = c->stream;
  // the smoothing weights, normalised to sum 1 (host, FP64)
  const int R = rule->sigma > 0.0 ? (int)std::ceil(3.0 * rule->sigma) : 0;
  std::vector<double> w(2 * R + 1, 1.0);
  if (R > 0) {
    double ws = 0.0;
    for (int j = -R; j <= R; ++j) {
      w[j + R] = std::exp(-(double)(j * j) / (2.0 * rule->sigma * rule->sigma));
      ws += w[j + R];
    }
    for (double& x : w) x /= ws;
  }
  long long* Q = (long long*)dalloc(c, sizeof(long long) * m.V);
  double* rho = (double*)dalloc(c, sizeof(double) * m.V);
  double* tmp = (double*)dalloc(c, sizeof(double) * m.V);
  double* ev = (double*)dalloc(c, sizeof(double) * m.V);
  double* wd = (double*)dalloc(c, sizeof(double) * (w.size() + 1));
  memd_status s = MEMD_OK;
  if (!Q || !rho || !tmp || !ev || !wd) {
    s = fail(c, MEMD_ERR_OOM, "salt density scratch");
  } else if (cudaMemcpyAsync(wd, w.data(), sizeof(double) * w.size(), cudaMemcpyHostToDevice, st) !=
             cudaSuccess) {
    s = fail(c, MEMD_ERR_CUDA, "smoothing weights");
  } else {
    launch_cic_abs(m, c->P, Q, st);
    launch_salt_eps(m, Q, rho, tmp, wd, R, rule->sigma, c->red, wd + w.size(), r4, ev, st);
    if (cudaGetLastError() != cudaSuccess) s = fail(c, MEMD_ERR_CUDA, "salt density kernels");
  }
  if (s == MEMD_OK && eps_out &&
      (cudaMemcpyAsync(eps_out, ev, sizeof(double) * m.V, cudaMemcpyDeviceToHost, st) != cudaSuccess ||
       cudaStreamSynchronize(st) != cudaSuccess))
    s = fail(c, MEMD_ERR_CUDA, "eps download");
  if (s == MEMD_OK) {
    memd_eps_profile e{};
    e.kind = MEMD_EPS_VERTICES;
    s = set_eps_impl(c, &e, relax_field, ev);
  }
  dfree(c, Q);
  dfree(c, rho);
  dfree(c, tmp);
  dfree(c, ev);
  dfree(c, wd);
  return s;
}

static memd_status set_eps_impl(memd_ctx* c, const memd_eps_profile* eps, int32_t relax_field,
                                const double* dev_values) {
  const cudaStream_t st = c->stream;
  if (c->initialised) {
    const memd_status fe = memd_flush(c);
    if (fe != MEMD_OK) return fe;
  }
  drop_graphs(c);
  harvest_timing(c);
  CK(cudaStreamSynchronize(st));
  memd_status s = setup_eps(c, eps, dev_values);
  if (s != MEMD_OK) return s;
  c->gen += 1;  // batches holding this context rebuild their tables
  if (!c->initialised) return MEMD_OK;
  if (relax_field) {
    const Mesh& m = c->mesh;
    double* D64 = (double*)dalloc(c, 3 * m.V * sizeof(double));
    if (!D64) return fail(c, MEMD_ERR_OOM, "relaxation field");
    const double scale = std::ldexp(1.0, -48) / (m.a * m.a);
    launch_dipole(m, c->P, c->ds, st);
    launch_ledger_sums(m, c->Lg, c->ds, st);
    launch_init_D(m, D64, c->Lg, c->ds, scale, c->Vbox, st);
    if (c->psi) {
      int its = 0;
      const memd_status ms = mg_relax(c, D64, c->psi, c->eps_eff_inv,
                                      std::min(c->relax_tol, 1e-12), c->relax_maxit, &its);
      if (ms != MEMD_OK) {
        cudaGetLastError();
        launch_init_D(m, D64, c->Lg, c->ds, scale, c->Vbox, st);
      }
    }
    s = relax(c, D64, c->relax_tol, c->relax_maxit);
    if (s == MEMD_OK) {
      launch_cast(c->prec, c->D(), D64, 3 * m.V, st);
      if (cudaMemsetAsync(c->B(), 0, 3 * m.V * esz(c), st) != cudaSuccess)
        s = fail(c, MEMD_ERR_CUDA, "memset");
    }
    dfree(c, D64);
    if (s != MEMD_OK) return s;
  }
  return memd_compute_forces(c);
}

memd_status memd_get_setup(memd_ctx* c, double* inv_eps, double* G8, double* eps_eff_inv) {
  if (!c) return MEMD_ERR_INVALID;
  CK(cudaSetDevice(c->device));
  if (inv_eps)
    CK(cudaMemcpyAsync(inv_eps, c->ie64, 3 * c->mesh.V * sizeof(double), cudaMemcpyDeviceToHost,
                       c->stream));
  CK(cudaStreamSynchronize(c->stream));
  if (G8) std::memcpy(G8, c->G, sizeof(c->G));
  if (eps_eff_inv) std::memcpy(eps_eff_inv, c->Minv, sizeof(c->Minv));
  return MEMD_OK;
}

memd_status memd_get_kernel_stats(memd_ctx* c, memd_kernel_stats* out) {
  if (!c || !out) return MEMD_ERR_INVALID;
  harvest_timing(c);
  out->field_ms = c->field_ms;
  out->field_launches = c->field_launches;
  // the fused update reads D, 1/eps, B and writes D', B' (15 values a site)
  const double e = (double)esz(c);
  out->field_bytes = 15.0 * e * (double)c->mesh.V;
  // the single launch also moves each particle's state once: x, v, Ft, img
  // read and written, F and the move written, q, m, h, sigma read, and the
  // 12 links of its cell (D, 1/eps, 1/eps FP64) read: 460 bytes
  if (c->coop) out->field_bytes += 460.0 * (double)c->P.n;
  out->launches_per_step = c->coop ? 1 : (c->P.n > 0 ? 4 : 2);
  out->step_single = c->coop ? 1 : 0;
  out->field_tx = 32;
  out->field_tma = c->fcfg.tma;
  out->field_ty = c->fcfg.ty;
  out->field_zchunk = c->fcfg.zchunk;
  out->field_site = c->fcfg.site;
  out->field_rows = c->fcfg.rows;
  return MEMD_OK;
}

memd_status memd_reset_kernel_stats(memd_ctx* c) {
  if (!c) return MEMD_ERR_INVALID;
  harvest_timing(c);
  c->field_ms = 0;
  c->field_launches = 0;
  return MEMD_OK;
}

memd_status memd_synchronize(memd_ctx* c) {
  if (!c) return MEMD_ERR_INVALID;
  CK(cudaSetDevice(c->device));
  harvest_timing(c);
  CK(cudaStreamSynchronize(c->stream));
  return check_err(c);
}

}  // extern "C"
