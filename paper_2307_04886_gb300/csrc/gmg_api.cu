// extern "C" entry points of libgmg (declared in include/gmg.h).
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstdlib>
#include <new>
#include <vector>
#include <string>

#include "gmg_cycle.cuh"

namespace gmg {
extern thread_local std::string g_last_error;

static bool is_pcg(int mode) { return mode == GMG_FP32_PCG || mode == GMG_FP64_PCG; }

static gmg_status check_handle(gmg_handle h) {
  if (!h) {
    set_error("null handle");
    return GMG_ERR_INVALID_ARG;
  }
  GMG_CK(cudaSetDevice(h->device));
  return GMG_OK;
}

// Runs one iteration body, from a captured graph when enabled.
static gmg_status run_body(gmg_ctx* c, int mode, int seg, cudaStream_t s) {
  if (!c->opt.use_graphs) return iteration_body(c, mode, seg, s);
  const int key = mode * 2 + seg;
  if (!c->graphs[key]) {
    if (!c->g_stream) GMG_CK(cudaStreamCreateWithFlags(&c->g_stream, cudaStreamNonBlocking));
    cudaGraph_t g = nullptr;
    const uint64_t before = g_launches;
    GMG_CK(cudaStreamBeginCapture(c->g_stream, cudaStreamCaptureModeThreadLocal));
    gmg_status st = iteration_body(c, mode, seg, c->g_stream);
    cudaError_t e = cudaStreamEndCapture(c->g_stream, &g);
    c->graph_kernels[key] = g_launches - before;  // captured, not yet run
    g_launches = before;
    if (st != GMG_OK) {
      if (g) cudaGraphDestroy(g);
      return st;
    }
    GMG_CK(e);
    cudaError_t ei = cudaGraphInstantiate(&c->graphs[key], g, 0);
    cudaGraphDestroy(g);
    GMG_CK(ei);
  }
  GMG_CK(cudaGraphLaunch(c->graphs[key], s));
  g_launches += c->graph_kernels[key];
  return GMG_OK;
}

static gmg_status fetch_scalars(gmg_ctx* c, cudaStream_t s) {
  GMG_CK(cudaMemcpyAsync(c->h_scal, c->scal, 8 * sizeof(double), cudaMemcpyDeviceToHost, s));
  GMG_CK(cudaStreamSynchronize(s));
  if (c->prof && c->prof_pending) {  // the last cycle's events have completed
    float a = 0, b = 0, v = 0;
    GMG_CK(cudaEventElapsedTime(&a, c->ev[0], c->ev[1]));
    GMG_CK(cudaEventElapsedTime(&b, c->ev[2], c->ev[3]));
    GMG_CK(cudaEventElapsedTime(&v, c->ev[4], c->ev[5]));
    c->prof_acc[0] += a + b;
    c->prof_acc[1] += (double)c->prof_gs;
    c->prof_acc[2] += v;
    c->prof_acc[3] += 1;
    for (int l = 0; l < c->nlev && (int)c->lev_ev.size() >= 6 * c->nlev; ++l) {
      cudaEvent_t* E = &c->lev_ev[6 * l];
      double* acc = &c->lev_acc[4 * l];
      float t = 0.f;
      if (c->lev_kind[l] == 1) {
        float p0 = 0, p1 = 0, t0 = 0, t1 = 0;
        GMG_CK(cudaEventElapsedTime(&p0, E[0], E[1]));
        GMG_CK(cudaEventElapsedTime(&p1, E[4], E[5]));
        GMG_CK(cudaEventElapsedTime(&t0, E[1], E[2]));
        GMG_CK(cudaEventElapsedTime(&t1, E[3], E[4]));
        acc[0] += p0 + p1;
        acc[1] += c->lev_gs[l];
        acc[2] += t0 + t1;
      }
      if (c->lev_kind[l] == 3) {  // cluster level: its two launches hold the sweeps and the transfers
        float p0 = 0, p1 = 0;
        GMG_CK(cudaEventElapsedTime(&p0, E[0], E[1]));
        GMG_CK(cudaEventElapsedTime(&p1, E[3], E[5]));
        acc[0] += p0 + p1;
        acc[1] += c->lev_gs[l];
      }
      if (c->lev_kind[l] != 0) {
        GMG_CK(cudaEventElapsedTime(&t, E[0], E[5]));
        acc[3] += t;
      }
    }
    c->prof_pending = false;
  }
  return GMG_OK;
}

static gmg_status run_cycle_body(gmg_ctx* c, int mode, int seg, cudaStream_t s) {
  GMG_TRY(run_body(c, mode, seg, s));
  if (c->nlev > 1 && (!is_pcg(mode) || seg == 1)) c->prof_pending = c->prof;
  return GMG_OK;
}

// Destroys every captured graph (their launch shapes or event nodes are stale).
static void drop_graphs(gmg_ctx* c) {
  for (auto& g : c->graphs)
    if (g) {
      cudaGraphExecDestroy(g);
      g = nullptr;
    }
  for (int m = 0; m < 4; ++m) {
    if (c->loops[m]) cudaGraphExecDestroy(c->loops[m]);
    c->loops[m] = nullptr;
    c->loop_refused[m] = false;
  }
}

// Builds the device-side loop of `mode`: a graph holding one conditional
// WHILE node (condition 1 at every launch) whose body is captured from
// loop_body.  The body keeps its programmatic launch edges if the CUDA driver
// instantiates them inside a conditional body, else it is captured again in
// plain stream order; if neither instantiates, the mode keeps the host loop.
static gmg_status build_loop(gmg_ctx* c, int mode) {
  if (!c->g_stream) GMG_CK(cudaStreamCreateWithFlags(&c->g_stream, cudaStreamNonBlocking));
  for (int attempt = 0; attempt < 2 && !c->loops[mode]; ++attempt) {
    cudaGraph_t g = nullptr;
    GMG_CK(cudaGraphCreate(&g, 0));
    cudaGraphConditionalHandle h = 0;
    cudaGraphNodeParams np = {};
    cudaError_t e = cudaGraphConditionalHandleCreate(&h, g, 1, cudaGraphCondAssignDefault);
    if (e == cudaSuccess) {
      np.type = cudaGraphNodeTypeConditional;
      np.conditional.handle = h;
      np.conditional.type = cudaGraphCondTypeWhile;
      np.conditional.size = 1;
      cudaGraphNode_t node;
      e = cudaGraphAddNode(&node, g, nullptr, nullptr, 0, &np);
    }
    if (e == cudaSuccess) {
      const uint64_t before = g_launches;
      g_pdl_suspended = attempt == 1;
      e = cudaStreamBeginCaptureToGraph(c->g_stream, np.conditional.phGraph_out[0], nullptr, nullptr, 0,
                                        cudaStreamCaptureModeThreadLocal);
      gmg_status st = GMG_OK;
      if (e == cudaSuccess) {
        st = loop_body(c, mode, h, c->g_stream);
        cudaGraph_t body = nullptr;
        e = cudaStreamEndCapture(c->g_stream, &body);
      }
      g_pdl_suspended = false;
      c->loop_kernels[mode] = g_launches - before;
      g_launches = before;
      if (st != GMG_OK) {
        cudaGraphDestroy(g);
        return st;
      }
      if (e == cudaSuccess) e = cudaGraphInstantiate(&c->loops[mode], g, 0);
      if (e == cudaSuccess) c->loop_pdl[mode] = attempt == 0 && use_pdl();
    }
    cudaGraphDestroy(g);
    if (e != cudaSuccess) {
      cudaGetLastError();
      c->loops[mode] = nullptr;
    }
  }
  if (!c->loops[mode]) c->loop_refused[mode] = true;
  if (const char* e = std::getenv("GMG_VERBOSE"))
    if (e[0] == '1')
      std::fprintf(stderr, "gmg: device-side loop for mode %d: %s\n", mode,
                   !c->loops[mode] ? "refused, host loop" : c->loop_pdl[mode] ? "programmatic launches" : "plain stream order");
  return GMG_OK;
}

// Whether the iterations of `mode` run in the device-side loop: graphs on,
// no per-cycle timing (event nodes are not allowed in a conditional body),
// GMG_NO_DEVICE_LOOP unset, and the loop graph instantiated.
static gmg_status device_loop_ready(gmg_ctx* c, int mode, bool* ok) {
  static const bool off = [] {
    const char* e = std::getenv("GMG_NO_DEVICE_LOOP");
    return e && e[0] == '1';
  }();
  *ok = false;
  if (off || !c->opt.use_graphs || c->prof || c->loop_refused[mode]) return GMG_OK;
  if (!c->loops[mode]) GMG_TRY(build_loop(c, mode));
  *ok = c->loops[mode] != nullptr;
  return GMG_OK;
}

// Runs the device-side loop from iteration *k until k_iter_check stops it;
// returns the new iteration count in *k, the scalars in h_scal and the
// loop's residual history in info->history.
static gmg_status run_loop(gmg_ctx* c, int mode, double tol, int* k, gmg_solve_info* info, cudaStream_t s) {
  const int it[2] = {*k, c->opt.max_iter};
  GMG_CK(cudaMemcpyAsync(c->scal + S_TOL, &tol, sizeof(double), cudaMemcpyHostToDevice, s));
  GMG_CK(cudaMemcpyAsync(c->dloop, it, sizeof(it), cudaMemcpyHostToDevice, s));
  GMG_CK(cudaGraphLaunch(c->loops[mode], s));
  int* hk = reinterpret_cast<int*>(c->h_scal + 40);
  GMG_CK(cudaMemcpyAsync(hk, c->dloop, sizeof(int), cudaMemcpyDeviceToHost, s));
  GMG_TRY(fetch_scalars(c, s));
  const int k1 = *hk;
  if (k1 <= *k || k1 > c->opt.max_iter) {
    set_error("device loop: iteration counter out of range");
    return GMG_ERR_CUDA;
  }
  g_launches += (uint64_t)(k1 - *k) * c->loop_kernels[mode];
  if (info && info->history && *k + 1 < info->history_cap) {
    const int last = std::min(k1, info->history_cap - 1);
    GMG_CK(cudaMemcpy(info->history + *k + 1, c->dhist + *k + 1, sizeof(double) * (size_t)(last - *k),
                      cudaMemcpyDeviceToHost));
  }
  *k = k1;
  return GMG_OK;
}

// Copies an n-vector in caller numbering (host or device) into the permuted
// device vector `dst` of level l.
static gmg_status load_vec(gmg_ctx* c, int l, const double* src, int mem, double* dst, double* stage,
                           cudaStream_t s) {
  Level& L = c->L[l];
  if (mem == GMG_MEM_HOST) {
    GMG_CK(cudaMemcpyAsync(stage, src, sizeof(double) * (size_t)L.n, cudaMemcpyHostToDevice, s));
    src = stage;
  }
  return launch_gather(L.n, L.perm, src, dst, s);
}

static gmg_status store_vec(gmg_ctx* c, int l, const double* src, double* dst, int mem, double* stage,
                            cudaStream_t s) {
  Level& L = c->L[l];
  if (mem == GMG_MEM_HOST) {
    GMG_TRY(launch_scatter(L.n, L.perm, src, stage, s));
    GMG_CK(cudaMemcpyAsync(dst, stage, sizeof(double) * (size_t)L.n, cudaMemcpyDeviceToHost, s));
    GMG_CK(cudaStreamSynchronize(s));
    return GMG_OK;
  }
  return launch_scatter(L.n, L.perm, src, dst, s);
}

}  // namespace gmg

using namespace gmg;

extern "C" {

void gmg_default_options(gmg_options* opt) {
  if (!opt) return;
  opt->precision = GMG_FP32_REFINE;
  opt->nu_pre = 2;
  opt->nu_post = 2;
  opt->max_iter = 100;
  opt->post_forward = 0;
  opt->use_graphs = 1;
}

const char* gmg_status_string(gmg_status s) {
  switch (s) {
    case GMG_OK: return "ok";
    case GMG_ERR_INVALID_ARG: return "invalid argument";
    case GMG_ERR_NOT_SPD: return "matrix not symmetric positive definite";
    case GMG_ERR_EMPTY_P_COLUMN: return "empty prolongation column";
    case GMG_ERR_CHOLESKY: return "coarsest Cholesky factorisation failed";
    case GMG_ERR_NOT_CONVERGED: return "not converged";
    case GMG_ERR_NONFINITE: return "non-finite value";
    case GMG_ERR_OOM: return "out of device memory";
    case GMG_ERR_CUDA: return "CUDA error";
    case GMG_ERR_TIMEOUT: return "device wait timed out";
    case GMG_ERR_TOO_LARGE: return "size limit exceeded";
  }
  return "unknown status";
}

const char* gmg_last_error(void) { return g_last_error.c_str(); }

uint64_t gmg_kernel_launches(void) { return g_launches; }

gmg_status gmg_destroy(gmg_handle h) {
  if (!h) return GMG_OK;
  cudaSetDevice(h->device);
  drop_graphs(h);
  if (h->g_stream) cudaStreamDestroy(h->g_stream);
  for (auto& e : h->ev)
    if (e) cudaEventDestroy(e);
  for (auto& e : h->lev_ev)
    if (e) cudaEventDestroy(e);
  if (h->h_scal) cudaFreeHost(h->h_scal);
  cudaDeviceSynchronize();
  if (h->inv_stream) cudaStreamDestroy(h->inv_stream);
  if (h->ev_gal) cudaEventDestroy(h->ev_gal);
  if (h->ev_inv) cudaEventDestroy(h->ev_inv);
  h->arena.release();
  delete h;
  return GMG_OK;
}

gmg_status gmg_setup(gmg_handle* h, const gmg_csr* A, int n_prolong, const gmg_prolong* P,
                     const int32_t* const* coloring, const gmg_options* opt, void* stream) {
  g_last_error.clear();
  if (!h || n_prolong < 0 || (n_prolong > 0 && !P)) {
    set_error("gmg_setup: null output handle or bad prolongation list");
    return GMG_ERR_INVALID_ARG;
  }
  *h = nullptr;
  gmg_ctx* c = new (std::nothrow) gmg_ctx();
  if (!c) return GMG_ERR_OOM;
  if (opt) c->opt = *opt;
  else gmg_default_options(&c->opt);
  if (const char* e = std::getenv("GMG_NO_GRAPHS"))  // profilers list graph nodes slowly
    if (e[0] == '1') c->opt.use_graphs = 0;
  if (c->opt.nu_pre < 0 || c->opt.nu_post < 0 || c->opt.max_iter < 0 || c->opt.precision < GMG_FP64 ||
      c->opt.precision > GMG_FP64_PCG) {
    set_error("gmg_setup: invalid options");
    delete c;
    return GMG_ERR_INVALID_ARG;
  }
  gmg_status st = setup_impl(c, A, n_prolong, P, coloring, (cudaStream_t)stream);
  if (st != GMG_OK) {
    std::string keep = g_last_error;
    gmg_destroy(c);
    g_last_error = keep;
    return st;
  }
  *h = c;
  return GMG_OK;
}

gmg_status gmg_set_values(gmg_handle h, const double* val, int mem, void* stream) {
  NvtxRange nv("gmg_set_values");
  GMG_TRY(check_handle(h));
  if (!val) {
    set_error("gmg_set_values: null values");
    return GMG_ERR_INVALID_ARG;
  }
  cudaStream_t s = (cudaStream_t)stream;
  Level& L0 = h->L[0];
  GMG_TRY(join_inverse(h, s, false));  // a previous refresh's inverse still reads the level values
  GMG_CK(cudaMemcpyAsync(L0.csr_val, val, sizeof(double) * (size_t)L0.nnz,
                         mem == GMG_MEM_HOST ? cudaMemcpyHostToDevice : cudaMemcpyDeviceToDevice, s));
  return numeric_setup(h, s, true);
}

gmg_status gmg_solve(gmg_handle h, const double* b, double* x, double tol, int mem, gmg_solve_info* info,
                     void* stream) {
  NvtxRange nv("gmg_solve");
  GMG_TRY(check_handle(h));
  if (!b || !x || !(tol >= 0.0) || (mem != GMG_MEM_HOST && mem != GMG_MEM_DEVICE)) {
    set_error("gmg_solve: null vector, negative tolerance or bad memory kind");
    return GMG_ERR_INVALID_ARG;
  }
  gmg_ctx* c = h;
  cudaStream_t s = (cudaStream_t)stream;
  Level& L0 = c->L[0];
  const int64_t n = L0.n;
  GMG_TRY(load_vec(c, 0, b, mem, c->bs, c->io, s));
  GMG_TRY(load_vec(c, 0, x, mem, c->xs, c->io2, s));
  GMG_TRY(norm_b(c, s));
  GMG_TRY(outer_residual_norm(c, s));
  GMG_TRY(fetch_scalars(c, s));
  const double nb = std::sqrt(c->h_scal[S_NB2]);
  int k = 0;
  double rel = 0.0;
  gmg_status st = GMG_ERR_NOT_CONVERGED;
  auto record = [&](int kk, double v) {
    if (info && info->history && kk < info->history_cap) info->history[kk] = v;
  };
  if (!std::isfinite(nb)) {
    set_error("gmg_solve: non-finite right-hand side");
    st = GMG_ERR_NONFINITE;
  } else if (nb == 0.0) {
    GMG_CK(cudaMemsetAsync(c->xs, 0, sizeof(double) * (size_t)n, s));
    record(0, 0.0);
    st = GMG_OK;
  } else {
    rel = std::sqrt(c->h_scal[S_RR]) / nb;
    record(0, rel);
    const int mode = c->nlev == 1 ? GMG_FP64 : c->opt.precision;
    if (!std::isfinite(rel)) {
      set_error("gmg_solve: non-finite initial residual");
      st = GMG_ERR_NONFINITE;
    } else {
      // a CG start joins a pending coarsest inverse right before its first
      // coarse solve (its down-leg overlaps the inverse); the other modes
      // join before their first iteration
      if (!is_pcg(mode)) GMG_TRY(join_inverse(c, s, false));
      if (is_pcg(mode)) GMG_TRY(pcg_start(c, mode, s));
      bool fresh = true;  // CG: no step since the (re)start
      while (k < c->opt.max_iter) {
        bool dev = false;
        if (!(is_pcg(mode) && fresh)) GMG_TRY(device_loop_ready(c, mode, &dev));
        if (dev) {
          GMG_TRY(run_loop(c, mode, tol, &k, info, s));
        } else {
          if (is_pcg(mode) && !fresh) GMG_TRY(run_cycle_body(c, mode, 1, s));
          GMG_TRY(run_cycle_body(c, mode, 0, s));
          GMG_TRY(fetch_scalars(c, s));
          ++k;
        }
        fresh = false;
        rel = std::sqrt(c->h_scal[S_RR]) / nb;
        if (!std::isfinite(rel)) {
          set_error("gmg_solve: iterate became non-finite");
          st = GMG_ERR_NONFINITE;
          break;
        }
        if (rel <= tol && is_pcg(mode)) {  // confirm on the true residual
          GMG_TRY(outer_residual_norm(c, s));
          GMG_TRY(fetch_scalars(c, s));
          rel = std::sqrt(c->h_scal[S_RR]) / nb;
          record(k, rel);
          if (rel <= tol) {
            st = GMG_OK;
            break;
          }
          GMG_TRY(pcg_start(c, mode, s));  // restart from the current iterate
          fresh = true;
          continue;
        }
        if (!dev) record(k, rel);  // the device loop wrote its own history
        if (rel <= tol) {
          st = GMG_OK;
          break;
        }
      }
      if (st == GMG_ERR_NOT_CONVERGED) set_error("gmg_solve: max_iter reached");
    }
  }
  GMG_TRY(store_vec(c, 0, c->xs, x, mem, c->io2, s));
  if (info) {
    info->iters = k;
    info->rel_res = rel;
  }
  GMG_TRY(inverse_status(c, s));  // the pivot check of an inverse this solve joined
  GMG_TRY(cluster_level_status(c, s));
  return st;
}

gmg_status gmg_profile(gmg_handle h, int enable) {
  GMG_TRY(check_handle(h));
  if ((enable != 0) == h->prof) return GMG_OK;
  if (enable && !h->ev[0])
    for (auto& e : h->ev) GMG_CK(cudaEventCreate(&e));
  if (enable && h->lev_ev.empty()) {
    h->lev_ev.assign(6 * h->nlev, nullptr);
    for (auto& e : h->lev_ev) GMG_CK(cudaEventCreate(&e));
    h->lev_kind.assign(h->nlev, 0);
    h->lev_gs.assign(h->nlev, 0);
    h->lev_acc.assign(4 * h->nlev, 0.0);
  }
  drop_graphs(h);  // re-capture with or without the event nodes
  h->prof = enable != 0;
  h->prof_pending = false;
  return GMG_OK;
}

gmg_status gmg_profile_read(gmg_handle h, double* out) {
  if (!h || !out) return GMG_ERR_INVALID_ARG;
  for (int k = 0; k < 4; ++k) {
    out[k] = h->prof_acc[k];
    h->prof_acc[k] = 0.0;
  }
  return GMG_OK;
}

gmg_status gmg_profile_levels(gmg_handle h, double* out) {
  if (!h || !out) return GMG_ERR_INVALID_ARG;
  const bool have = (int)h->lev_acc.size() >= 4 * h->nlev;
  for (int k = 0; k < 4 * h->nlev; ++k) {
    out[k] = have ? h->lev_acc[k] : 0.0;
    if (have) h->lev_acc[k] = 0.0;
  }
  return GMG_OK;
}

// Makes a new warps-per-row choice take effect: captured cycles hold the old
// launch shapes.
static gmg_status apply_lanes(gmg_handle h) {
  drop_graphs(h);
  return GMG_OK;
}

gmg_status gmg_autotune(gmg_handle h, int* lanes_out, void* stream) {
  GMG_TRY(check_handle(h));
  // The sweeps are timed as they run in a solve: captured in a CUDA graph with
  // programmatic launches, where the cost of a phase depends on its CTA count
  // and dependent loads rather than on the host's launch rate.
  GMG_CK(cudaStreamSynchronize((cudaStream_t)stream));
  if (!h->g_stream) GMG_CK(cudaStreamCreateWithFlags(&h->g_stream, cudaStreamNonBlocking));
  cudaStream_t cs = h->g_stream;
  cudaEvent_t e0, e1;
  GMG_CK(cudaEventCreate(&e0));
  GMG_CK(cudaEventCreate(&e1));
  gmg_status st = GMG_OK;
  const uint64_t launches_before = g_launches;
  for (int l = 0; l + 1 < h->nlev && st == GMG_OK; ++l) {
    Level& L = h->L[l];
    const int keep = L.lanes;
    float best_ms = 1e30f;
    int best = keep;
    if (cudaMemsetAsync(L.x32, 0, sizeof(float) * (size_t)L.n, cs) != cudaSuccess ||
        cudaMemsetAsync(L.b32, 0, sizeof(float) * (size_t)L.n, cs) != cudaSuccess) {
      st = GMG_ERR_CUDA;
      break;
    }
    for (int G : {1, 2, 4, 8}) {
      L.lanes = G;
      cudaGraph_t g = nullptr;
      cudaGraphExec_t ge = nullptr;
      if (cudaStreamBeginCapture(cs, cudaStreamCaptureModeThreadLocal) != cudaSuccess) {
        st = GMG_ERR_CUDA;
        break;
      }
      for (int sweep = 0; sweep < 4 && st == GMG_OK; ++sweep)
        for (int k = 0; k < L.ncolor && st == GMG_OK; ++k) st = launch_gs_colour<float>(L, k, L.b32, L.x32, cs);
      const cudaError_t ec = cudaStreamEndCapture(cs, &g);
      if (st == GMG_OK && ec == cudaSuccess && cudaGraphInstantiate(&ge, g, 0) == cudaSuccess) {
        float ms = 0.f;
        cudaGraphLaunch(ge, cs);  // warm-up
        cudaEventRecord(e0, cs);
        for (int rep = 0; rep < 3; ++rep) cudaGraphLaunch(ge, cs);
        cudaEventRecord(e1, cs);
        if (cudaEventSynchronize(e1) != cudaSuccess) st = GMG_ERR_CUDA;
        cudaEventElapsedTime(&ms, e0, e1);
        if (st == GMG_OK && ms < best_ms) {
          best_ms = ms;
          best = G;
        }
      } else if (st == GMG_OK) {
        set_error("gmg_autotune: graph capture of the sweeps failed");
        st = GMG_ERR_CUDA;
      }
      if (ge) cudaGraphExecDestroy(ge);
      if (g) cudaGraphDestroy(g);
    }
    L.lanes = st == GMG_OK ? best : keep;
    if (lanes_out) lanes_out[l] = L.lanes;
    // the residual covers every row at once: its own split, timed the same way
    const int rkeep = L.rlanes;
    float rbest_ms = 1e30f;
    int rbest = rkeep;
    for (int G : {1, 2, 4, 8}) {
      if (st != GMG_OK) break;
      L.rlanes = G;
      cudaGraph_t g = nullptr;
      cudaGraphExec_t ge = nullptr;
      if (cudaStreamBeginCapture(cs, cudaStreamCaptureModeThreadLocal) != cudaSuccess) {
        st = GMG_ERR_CUDA;
        break;
      }
      for (int rep = 0; rep < 4 && st == GMG_OK; ++rep) st = launch_residual<float>(L, L.x32, L.b32, L.r32, cs);
      const cudaError_t ec = cudaStreamEndCapture(cs, &g);
      if (st == GMG_OK && ec == cudaSuccess && cudaGraphInstantiate(&ge, g, 0) == cudaSuccess) {
        float ms = 0.f;
        cudaGraphLaunch(ge, cs);  // warm-up
        cudaEventRecord(e0, cs);
        for (int rep = 0; rep < 3; ++rep) cudaGraphLaunch(ge, cs);
        cudaEventRecord(e1, cs);
        if (cudaEventSynchronize(e1) != cudaSuccess) st = GMG_ERR_CUDA;
        cudaEventElapsedTime(&ms, e0, e1);
        if (st == GMG_OK && ms < rbest_ms) {
          rbest_ms = ms;
          rbest = G;
        }
      } else if (st == GMG_OK) {
        set_error("gmg_autotune: graph capture of the residuals failed");
        st = GMG_ERR_CUDA;
      }
      if (ge) cudaGraphExecDestroy(ge);
      if (g) cudaGraphDestroy(g);
    }
    L.rlanes = st == GMG_OK ? rbest : rkeep;
  }
  g_launches = launches_before;  // timing launches are not the caller's work
  cudaStreamSynchronize(cs);
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  if (st == GMG_OK) st = apply_lanes(h);
  return st;
}

gmg_status gmg_set_lanes(gmg_handle h, const int* lanes) {
  GMG_TRY(check_handle(h));
  if (!lanes) {
    set_error("gmg_set_lanes: null lanes");
    return GMG_ERR_INVALID_ARG;
  }
  for (int l = 0; l + 1 < h->nlev; ++l)
    if (lanes[l] != 1 && lanes[l] != 2 && lanes[l] != 4 && lanes[l] != 8) {
      set_error("gmg_set_lanes: level " + std::to_string(l) + " split " + std::to_string(lanes[l]) +
                " is not 1, 2, 4 or 8");
      return GMG_ERR_INVALID_ARG;
    }
  for (int l = 0; l + 1 < h->nlev; ++l) h->L[l].lanes = h->L[l].rlanes = lanes[l];
  return apply_lanes(h);
}

gmg_status gmg_num_levels(gmg_handle h, int* nlev) {
  if (!h || !nlev) return GMG_ERR_INVALID_ARG;
  *nlev = h->nlev;
  return GMG_OK;
}

gmg_status gmg_warnings(gmg_handle h, uint32_t* flags, double* max_dev) {
  if (!h || !flags) return GMG_ERR_INVALID_ARG;
  *flags = h->p_unity_dev > 1e-12 ? GMG_WARN_P_UNITY : 0u;
  if (max_dev) *max_dev = h->p_unity_dev;
  return GMG_OK;
}

gmg_status gmg_level_info(gmg_handle h, int l, int64_t* n, int64_t* nnz, int* ncolors) {
  if (!h || l < 0 || l >= h->nlev) return GMG_ERR_INVALID_ARG;
  if (n) *n = h->L[l].n;
  if (nnz) *nnz = h->L[l].nnz;
  if (ncolors) *ncolors = h->L[l].ncolor;
  return GMG_OK;
}

gmg_status gmg_level_path(gmg_handle h, int l, int* path) {
  if (!h || !path || l < 0 || l >= h->nlev) return GMG_ERR_INVALID_ARG;
  if (l == h->nlev - 1)
    *path = 3;
  else if (h->tail_l0 > 0 && l >= h->tail_l0)
    *path = 2;
  else if (h->clev.l > 0 && l == h->clev.l)
    *path = 1;
  else
    *path = 0;
  return GMG_OK;
}

gmg_status gmg_level_export(gmg_handle h, int l, int64_t* rowptr, int32_t* col, double* val, int32_t* color) {
  GMG_TRY(check_handle(h));
  if (l < 0 || l >= h->nlev) return GMG_ERR_INVALID_ARG;
  Level& L = h->L[l];
  GMG_CK(cudaDeviceSynchronize());
  if (rowptr) GMG_CK(cudaMemcpy(rowptr, L.csr_rowptr, sizeof(int64_t) * (size_t)(L.n + 1), cudaMemcpyDeviceToHost));
  if (col) GMG_CK(cudaMemcpy(col, L.csr_col, sizeof(int32_t) * (size_t)L.nnz, cudaMemcpyDeviceToHost));
  if (val) GMG_CK(cudaMemcpy(val, L.csr_val, sizeof(double) * (size_t)L.nnz, cudaMemcpyDeviceToHost));
  if (color) std::copy(L.h_color.begin(), L.h_color.end(), color);
  return GMG_OK;
}

// ---- single steps of Alg. 2 (device vectors, caller numbering) ----

static gmg_status to_level(gmg_ctx* c, int l, int fp32, const double* src, double* d64, float* d32,
                           cudaStream_t s) {
  GMG_TRY(launch_gather(c->L[l].n, c->L[l].perm, src, d64, s));
  if (fp32) GMG_TRY(launch_d2f(c->L[l].n, d64, d32, s));
  return GMG_OK;
}
static gmg_status from_level(gmg_ctx* c, int l, int fp32, double* d64, const float* d32, double* dst,
                             cudaStream_t s) {
  if (fp32) GMG_TRY(launch_f2d(c->L[l].n, d32, d64, s));
  return launch_scatter(c->L[l].n, c->L[l].perm, d64, dst, s);
}

gmg_status gmg_smooth(gmg_handle h, int l, int fp32, const double* b, double* x, int nsweep, int descending,
                      void* stream) {
  GMG_TRY(check_handle(h));
  if (l < 0 || l >= h->nlev || !b || !x || nsweep < 0) return GMG_ERR_INVALID_ARG;
  cudaStream_t s = (cudaStream_t)stream;
  Level& L = h->L[l];
  GMG_TRY(to_level(h, l, fp32, b, L.b64, L.b32, s));
  GMG_TRY(to_level(h, l, fp32, x, L.x64, L.x32, s));
  for (int it = 0; it < nsweep; ++it)
    for (int q = 0; q < L.ncolor; ++q) {
      const int k = descending ? L.ncolor - 1 - q : q;
      if (fp32) GMG_TRY(launch_gs_colour<float>(L, k, L.b32, L.x32, s));
      else GMG_TRY(launch_gs_colour<double>(L, k, L.b64, L.x64, s));
    }
  return from_level(h, l, fp32, L.x64, L.x32, x, s);
}

gmg_status gmg_residual(gmg_handle h, int l, int fp32, const double* x, const double* b, double* r, void* stream) {
  GMG_TRY(check_handle(h));
  if (l < 0 || l >= h->nlev || !b || !x || !r) return GMG_ERR_INVALID_ARG;
  cudaStream_t s = (cudaStream_t)stream;
  Level& L = h->L[l];
  GMG_TRY(to_level(h, l, fp32, b, L.b64, L.b32, s));
  GMG_TRY(to_level(h, l, fp32, x, L.x64, L.x32, s));
  if (fp32) GMG_TRY(launch_residual<float>(L, L.x32, L.b32, L.r32, s));
  else GMG_TRY(launch_residual<double>(L, L.x64, L.b64, L.r64, s));
  return from_level(h, l, fp32, L.r64, L.r32, r, s);
}

gmg_status gmg_restrict(gmg_handle h, int l, int fp32, const double* r, double* bc, void* stream) {
  GMG_TRY(check_handle(h));
  if (l < 0 || l + 1 >= h->nlev || !r || !bc) return GMG_ERR_INVALID_ARG;
  cudaStream_t s = (cudaStream_t)stream;
  Level& L = h->L[l];
  Level& C = h->L[l + 1];
  GMG_TRY(to_level(h, l, fp32, r, L.r64, L.r32, s));
  if (fp32) GMG_TRY(launch_restrict<float>(L, L.r32, C.b32, C.x32, s));
  else GMG_TRY(launch_restrict<double>(L, L.r64, C.b64, C.x64, s));
  return from_level(h, l + 1, fp32, C.b64, C.b32, bc, s);
}

gmg_status gmg_prolong_add(gmg_handle h, int l, int fp32, const double* u, double* x, void* stream) {
  GMG_TRY(check_handle(h));
  if (l < 0 || l + 1 >= h->nlev || !u || !x) return GMG_ERR_INVALID_ARG;
  cudaStream_t s = (cudaStream_t)stream;
  Level& L = h->L[l];
  Level& C = h->L[l + 1];
  GMG_TRY(to_level(h, l + 1, fp32, u, C.x64, C.x32, s));
  GMG_TRY(to_level(h, l, fp32, x, L.x64, L.x32, s));
  if (fp32) GMG_TRY(launch_prolong<float>(L, C.x32, L.x32, s));
  else GMG_TRY(launch_prolong<double>(L, C.x64, L.x64, s));
  return from_level(h, l, fp32, L.x64, L.x32, x, s);
}

gmg_status gmg_coarse_solve(gmg_handle h, int fp32, const double* b, double* x, void* stream) {
  GMG_TRY(check_handle(h));
  if (!b || !x) return GMG_ERR_INVALID_ARG;
  cudaStream_t s = (cudaStream_t)stream;
  GMG_TRY(join_inverse(h, s, true));
  const int l = h->nlev - 1;
  Level& C = h->L[l];
  GMG_TRY(to_level(h, l, fp32, b, C.b64, C.b32, s));
  if (fp32) GMG_TRY(launch_coarse<float>(h, C.b32, C.x32, s));
  else GMG_TRY(launch_coarse<double>(h, C.b64, C.x64, s));
  return from_level(h, l, fp32, C.x64, C.x32, x, s);
}

gmg_status gmg_vcycle(gmg_handle h, int fp32, const double* b, double* x, void* stream) {
  GMG_TRY(check_handle(h));
  if (!b || !x) return GMG_ERR_INVALID_ARG;
  cudaStream_t s = (cudaStream_t)stream;
  GMG_TRY(join_inverse(h, s, true));
  Level& L = h->L[0];
  GMG_TRY(to_level(h, 0, fp32, b, L.b64, L.b32, s));
  GMG_TRY(to_level(h, 0, fp32, x, L.x64, L.x32, s));
  if (fp32) GMG_TRY(vcycle<float>(h, 0, s));
  else GMG_TRY(vcycle<double>(h, 0, s));
  return from_level(h, 0, fp32, L.x64, L.x32, x, s);
}

}  // extern "C"
