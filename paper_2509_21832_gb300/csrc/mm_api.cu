// Host side of the C ABI declared in include/mmkfvs.h: validation, device state, launch order of
// one time step (Section 5 of Rossmanith & Sar, arXiv 2509.21832: prims of Q^n, micro x sweep,
// micro y sweep + relaxation + heat flux, macro collision/x transport, macro y transport/
// collision), per-kernel event timing and error latching.
#include <algorithm>
#include <cmath>
#include <cstdint>
#include <cstdio>
#include <cstring>
#include <string>
#include <utility>
#include <vector>

#include "mm_internal.cuh"

using namespace mmk;

namespace {

const char* const kKernelNames[] = {
    "prims",    "micro_x",          "micro_y",   "micro_y_wall",   "macro_x1",
    "macro_x2", "macro_y",          "h_unpack",  "micro_fused",    "closure_features",
    "mlp_infer", "closure_decide",  "closure_lists", "closure_ghat", "closure_predict",
    "prims_uT"};
constexpr int kNumKernels = 16;
enum {
  T_PRIMS = 0, T_MICRO_X, T_MICRO_Y, T_MICRO_YW, T_MACRO_X1, T_MACRO_X2, T_MACRO_Y, T_HUNPACK,
  T_MICRO_FUSED, T_CL_FEATURES, T_MLP, T_CL_DECIDE, T_CL_LISTS, T_CL_GHAT, T_CL_PREDICT,
  T_PRIMS_UT
};

struct TimedLaunch {
  int kind;
  cudaEvent_t a, b;
};

}  // namespace

struct mm_ctx {
  mm_grid grid;
  mm_params params;
  KGrid kg;
  KParams kp;
  MicroShape ms;
  cudaStream_t stream = nullptr;
  int device = 0;
  bool fp32 = false;
  size_t nphase = 0, ncell = 0;
  void* G = nullptr;     // G^n (and G^{n+1} after the step)
  void* Gs = nullptr;    // FP64: G* (scratch); FP32: the other buffer of the ping-pong pair
  void* Gexp = nullptr;  // FP32 with diffuse walls: G* exported for the wall kernel
  int nseg = 1;          // FP32: row segments of the fused kernel
  double* Q = nullptr;
  double* macro = nullptr;  // Q*, Q**, half fluxes, boundary fluxes (scratch)
  MacroBufs mb{};
  double* H = nullptr;
  float* Hf = nullptr;      // FP32-g heat flux as (hi, lo) pairs
  double* prim = nullptr;
  float* primf = nullptr;  // FP32 copies of the per-cell coefficients (FP32-g path)
  // FP64 with one row per pass: raw row sums of G [cell][3][nv1], kept current with G (left by
  // the y sweeps, formed whenever G is set otherwise) for the x sweep
  double* rmom = nullptr;
  double* etab = nullptr;  // e1, e2 of every cell, from the x sweep to the y sweep (FP64 g)
  int* err = nullptr;
  int* wall_cells = nullptr;
  int n_wall = 0;
  bool have_state = false;
  // mm_create_borrowed: Q, G and the scratch buffers belong to the caller; user_G is the caller's
  // g buffer, which holds the state whenever a call returns (FP32 g ping-pongs inside mm_step)
  bool borrowed = false;
  void* user_G = nullptr;
  std::string last_error;
  // learned closure (FP64 contexts): network, threshold and per-cell buffers
  const mm_mlp* mlp = nullptr;
  double closure_thr = 0.0;
  float* cX = nullptr;                   // features [nc][39]
  float* cY = nullptr;                   // network outputs [nc][4]
  double* caux = nullptr;                // H_CE [4][nc], scale [nc]
  unsigned char* cflags = nullptr;       // 1: closure cell in the last hybrid step
  unsigned char* cvalid = nullptr;       // 1: g of the cell is current (micro-updated last step)
  bool cstale = false;                   // closure switched off: reset non-current g first
  int* clists = nullptr;                 // x-sweep, y-sweep and refresh cell lists [3][nc]
  int* ccounts = nullptr;                // their lengths [3]
  unsigned long long* cstat = nullptr;   // closure cells summed over hybrid steps
  long long closure_steps = 0;
  // fallback at low closure fractions: every cl_period-th step is a hybrid step whose closure
  // count decides the next cl_period - 1 steps (plain when below cl_min_frac of the cells)
  double cl_min_frac = 0.25;
  int cl_period = 16;
  int cl_left = 0;                        // steps before the next evaluation
  bool cl_plain = false;                  // the steps until then run the plain step
  unsigned long long cl_seen = 0;         // cstat at the last evaluation
  unsigned long long* cl_host = nullptr;  // pinned copy of cstat
  long long fallback_steps = 0;           // plain steps run in place of hybrid ones
  int blocks_x = 0, blocks_y = 0, blocks_g = 0;
  // manufactured-solution harness (FP64 contexts)
  bool mms = false;
  double mms_t = 0.0;                    // time t^n of the next step's source
  double* mms_phi = nullptr;             // velocity tables phi, Gcal/F [nv]
  double* mms_gam = nullptr;
  double* mms_src_g = nullptr;           // source term of g^{n+1} (layout of G)
  double* mms_src_q = nullptr;           // int (1, v, v v) S dv [6][ny][nx]
  // mm_step_host: streams for the row-chunk copies of g and for the x sweeps; events per chunk
  cudaStream_t cstream = nullptr, xstream = nullptr, ystream = nullptr;
  // FP32 g: the collision half step and x half fluxes of Q^n run on mstream beside the
  // phase-space kernel (they need only Q^n); ev_fork marks Q^n, ev_x1 their end
  cudaStream_t mstream = nullptr;
  cudaEvent_t ev_fork = nullptr, ev_x1 = nullptr;
  std::vector<cudaEvent_t> chunk_events;
  bool timing = false;
  std::vector<TimedLaunch> pending;
  std::vector<cudaEvent_t> free_events;
  double acc_ms[kNumKernels] = {0};
  long long acc_n[kNumKernels] = {0};
};

namespace {

mm_status fail(mm_ctx* c, mm_status s, const std::string& msg) {
  if (c) c->last_error = msg;
  return s;
}

mm_status cuda_fail(mm_ctx* c, cudaError_t e, const char* what) {
  return fail(c, MM_ERR_CUDA, std::string(what) + ": " + cudaGetErrorString(e));
}

std::string validate(const mm_grid* g, const mm_params* p) {
  if (!g || !p) return "null grid or params";
  if (g->nx < 1 || g->ny < 1) return "nx and ny must be >= 1";
  if (g->nv1 < 1 || g->nv2 < 1 || g->nv1 > 512 || g->nv2 > 1024)
    return "nv1 must be in 1..512 and nv2 in 1..1024";
  if (!(g->x1 > g->x0) || !(g->y1 > g->y0)) return "empty spatial box";
  if (!(g->v1max > g->v1min) || !(g->v2max > g->v2min)) return "empty velocity box";
  if (!(p->nu >= -1.0 && p->nu < 1.0)) return "nu must satisfy -1 <= nu < 1";
  if (p->tau_model < 0 || p->tau_model > 3) return "unknown tau model";
  if ((p->tau_model == MM_TAU_RHO || p->tau_model == MM_TAU_PRESSURE ||
       p->tau_model == MM_TAU_CONST) && !(p->tau0 > 0.0))
    return "tau0 must be > 0";
  if (p->precision != MM_PREC_FP64 && p->precision != MM_PREC_G_FP32) return "unknown precision";
  if (p->precision == MM_PREC_G_FP32 && g->nv1 > 32) return "MM_PREC_G_FP32 needs nv1 <= 32";
  if (p->precision == MM_PREC_G_FP32) {
    // the fused kernel keeps three rows of G* per warp in shared memory
    KGrid kg{};
    kg.nv1 = g->nv1;
    kg.nv2 = g->nv2;
    kg.v2min = g->v2min;
    kg.dv2 = (g->v2max - g->v2min) / g->nv2;
    if (fused_smem_f32(kg) > kMaxSmemPerCta)
      return "MM_PREC_G_FP32: the velocity mesh is too large for the fused kernel's shared memory";
  }
  for (int s = 0; s < 4; ++s) {
    if (p->bc[s] < 0 || p->bc[s] > 3) return "unknown boundary kind";
    if (p->bc[s] == MM_BC_DIFFUSE && !(p->wall_T[s] > 0.0)) return "diffuse wall needs wall_T > 0";
  }
  if ((p->bc[0] == MM_BC_PERIODIC) != (p->bc[1] == MM_BC_PERIODIC)) return "periodic x sides must be paired";
  if ((p->bc[2] == MM_BC_PERIODIC) != (p->bc[3] == MM_BC_PERIODIC)) return "periodic y sides must be paired";
  const bool specx = p->bc[0] == MM_BC_SPECULAR || p->bc[1] == MM_BC_SPECULAR;
  const bool specy = p->bc[2] == MM_BC_SPECULAR || p->bc[3] == MM_BC_SPECULAR;
  if (specx && std::fabs(g->v1min + g->v1max) > 1e-12 * (g->v1max - g->v1min))
    return "specular x walls need a velocity mesh symmetric in v1";
  if (specy && std::fabs(g->v2min + g->v2max) > 1e-12 * (g->v2max - g->v2min))
    return "specular y walls need a velocity mesh symmetric in v2";
  return "";
}

void destroy_events(mm_ctx* c) {
  for (auto& t : c->pending) {
    cudaEventDestroy(t.a);
    cudaEventDestroy(t.b);
  }
  c->pending.clear();
  for (auto e : c->free_events) cudaEventDestroy(e);
  c->free_events.clear();
}

cudaEvent_t take_event(mm_ctx* c) {
  if (!c->free_events.empty()) {
    cudaEvent_t e = c->free_events.back();
    c->free_events.pop_back();
    return e;
  }
  cudaEvent_t e;
  cudaEventCreate(&e);
  return e;
}

// Fold finished timed launches into the per-kernel totals (requires the stream to be idle).
void drain_timing(mm_ctx* c) {
  for (auto& t : c->pending) {
    float ms = 0.f;
    if (cudaEventElapsedTime(&ms, t.a, t.b) == cudaSuccess) {
      c->acc_ms[t.kind] += ms;
      c->acc_n[t.kind] += 1;
    }
    c->free_events.push_back(t.a);
    c->free_events.push_back(t.b);
  }
  c->pending.clear();
}

// A launch timed by events on the stream it runs on (the context stream unless given).
template <typename F>
void timed_on(mm_ctx* c, int kind, cudaStream_t st, F&& launch) {
  if (!c->timing) {
    launch();
    return;
  }
  if (c->pending.size() > 50000) {
    cudaDeviceSynchronize();
    drain_timing(c);
  }
  TimedLaunch t{kind, take_event(c), take_event(c)};
  cudaEventRecord(t.a, st);
  launch();
  cudaEventRecord(t.b, st);
  c->pending.push_back(t);
}

template <typename F>
void timed(mm_ctx* c, int kind, F&& launch) {
  timed_on(c, kind, c->stream, launch);
}

// The per-cell fields of Q^n (two kernels, each timed).
void enqueue_prims(mm_ctx* c, double dt, double eps, cudaStream_t s) {
  timed(c, T_PRIMS_UT, [&] { launch_prims_uT(c->Q, c->prim, c->kg, s); });
  timed(c, T_PRIMS, [&] {
    launch_prims(c->Q, c->prim, c->primf, c->kg, c->kp, dt, eps, c->err, s);
  });
}

mm_status check_device_errors(mm_ctx* c) {
  int h = 0;
  cudaError_t e = cudaMemcpyAsync(&h, c->err, sizeof(int), cudaMemcpyDeviceToHost, c->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
  if (e != cudaSuccess) return cuda_fail(c, e, "device error check");
  if (h & ERR_WAIT_TIMEOUT)
    return fail(c, MM_ERR_TIMEOUT, "a bounded device wait ran out (bulk copy into shared memory)");
  if (h) {
    char buf[160];
    std::snprintf(buf, sizeof buf,
                  "non-physical state met on the device (flags 0x%x: 1 prims of Q^n, 2 macro "
                  "update, 4 non-finite heat flux)", h);
    return fail(c, MM_ERR_NONPHYSICAL, buf);
  }
  return MM_OK;
}

template <typename Tg>
void enqueue_plain(mm_ctx* c, double dt, double eps) {
  Tg* G = static_cast<Tg*>(c->G);
  Tg* Gs = static_cast<Tg*>(c->Gs);
  const KGrid& g = c->kg;
  const KParams& p = c->kp;
  cudaStream_t s = c->stream;
  bool x1_side = false;
  if constexpr (sizeof(Tg) == sizeof(float)) {
    // (u1, u2, T) in FP64, then the FP32 coefficients of the phase-space kernels
    timed(c, T_PRIMS_UT, [&] { launch_prims_uT(c->Q, c->prim, c->kg, s); });
    timed(c, T_PRIMS, [&] {
      launch_prims_f32(c->Q, c->prim, c->primf, c->kg, c->kp, dt, eps, c->err, s);
    });
  } else {
    enqueue_prims(c, dt, eps, s);
  }
  if constexpr (sizeof(Tg) == sizeof(float)) {
    // macro x1 (collision half step and x half fluxes of Q^n) beside the phase-space kernel:
    // forked after the per-cell fields, so that it runs with the FP32 kernel rather than against
    // the FP64-bound fields kernel
    cudaError_t e = cudaSuccess;
    if (!c->mstream) e = cudaStreamCreateWithFlags(&c->mstream, cudaStreamNonBlocking);
    if (e == cudaSuccess && !c->ev_fork)
      e = cudaEventCreateWithFlags(&c->ev_fork, cudaEventDisableTiming);
    if (e == cudaSuccess && !c->ev_x1)
      e = cudaEventCreateWithFlags(&c->ev_x1, cudaEventDisableTiming);
    if (e == cudaSuccess) e = cudaEventRecord(c->ev_fork, s);
    if (e == cudaSuccess) e = cudaStreamWaitEvent(c->mstream, c->ev_fork, 0);
    if (e == cudaSuccess) {
      timed_on(c, T_MACRO_X1, c->mstream, [&] {
        launch_macro_x1(c->Q, c->mb, c->kg, c->kp, dt, eps, c->err, c->mstream);
      });
      x1_side = cudaEventRecord(c->ev_x1, c->mstream) == cudaSuccess;
    }
    if (!x1_side) cudaGetLastError();  // side stream unavailable: macro x1 runs in order below
  }
  const double* srcg = nullptr;
  const double* srcq = nullptr;
  if constexpr (sizeof(Tg) == sizeof(double)) {
    if (c->mms) {
      launch_mms_source(c->prim, c->mms_phi, c->mms_gam, c->mms_src_g, c->mms_src_q, g, p,
                        c->mms_t, dt, eps, c->grid.x0, c->grid.y0, s);
      srcg = c->mms_src_g;
      srcq = c->mms_src_q;
      c->mms_t += dt;
    }
    if (c->cstale) {  // after hybrid steps: g of closure cells to Ghat(Q^n) before a full step
      const int nc = (int)c->ncell;
      launch_closure_stale(c->cvalid, g, c->clists + 2 * nc, c->ccounts + 2, s);
      // (with the row sums of the new g)
      launch_closure_ghat(G, c->prim, g, dt, eps, c->ms, c->clists + 2 * nc, c->ccounts + 2,
                          c->blocks_g, s, c->rmom);
      c->cstale = false;
    }
  }
  if constexpr (sizeof(Tg) == sizeof(float)) {
    // fused streaming kernel: G -> Gs (ping-pong), wall cells from the exported G*
    float* Ge = static_cast<float*>(c->Gexp);
    timed(c, T_MICRO_FUSED, [&] {
      launch_micro_fused_f32(G, Gs, Ge, c->Hf, c->primf, g, p, dt, c->ms, c->nseg, c->err, s);
    });
    timed(c, T_HUNPACK, [&] { launch_h_unpack(c->Hf, c->H, g, eps, s); });
    if (c->n_wall > 0)
      timed(c, T_MICRO_YW, [&] {
        launch_wall_f32(Ge, Gs, c->H, c->Q, c->prim, c->wall_cells, c->n_wall, g, p, dt, eps,
                        c->err, s);
      });
    std::swap(c->G, c->Gs);
  } else {
    // the x sweep from the row sums of G (left by the previous y sweep, or formed when G was
    // set), for one row per pass
    if (c->rmom)
      timed(c, T_MICRO_X, [&] {
        launch_micro_x_rows<Tg>(G, Gs, c->prim, c->rmom, g, p, dt, c->ms, s, 0, -1, c->etab);
      });
    else
      timed(c, T_MICRO_X, [&] {
        launch_micro_x<Tg>(G, Gs, c->prim, g, p, dt, c->ms, s, 0, -1, c->etab);
      });
    timed(c, T_MICRO_Y, [&] {
      launch_micro_y<Tg>(Gs, G, c->H, c->prim, g, p, dt, eps, c->ms, c->err, s, srcg, 0, -1,
                         c->rmom, c->etab);
    });
    if (c->n_wall > 0)
      timed(c, T_MICRO_YW, [&] {
        launch_micro_y_wall<Tg>(Gs, G, c->H, c->prim, c->wall_cells, c->n_wall, g, p, dt, eps,
                                c->ms, c->err, s, c->rmom);
      });
  }
  if (x1_side) cudaStreamWaitEvent(s, c->ev_x1, 0);
  else timed(c, T_MACRO_X1, [&] { launch_macro_x1(c->Q, c->mb, g, p, dt, eps, c->err, s); });
  timed(c, T_MACRO_X2, [&] { launch_macro_x2(c->H, c->mb, g, p, dt, c->err, s); });
  timed(c, T_MACRO_Y, [&] { launch_macro_y(c->H, c->mb, c->Q, g, p, dt, eps, c->err, s, srcq); });
}

// Hybrid step with the learned closure (FP64): features, network and decision on every cell (one
// fused kernel), the work lists, g^n = Ghat(Q^n) on the cells the sweeps read whose g is not
// current, then the micro sweeps on the micro cells (x sweep also on their y neighbours).
void enqueue_hybrid(mm_ctx* c, double dt, double eps) {
  double* G = static_cast<double*>(c->G);
  double* Gs = static_cast<double*>(c->Gs);
  const KGrid& g = c->kg;
  const KParams& p = c->kp;
  cudaStream_t s = c->stream;
  const int nc = (int)c->ncell;
  enqueue_prims(c, dt, eps, s);
  timed(c, T_CL_PREDICT, [&] {
    launch_closure_predict(c->Q, c->prim, c->mlp, g, p, eps, dt, c->closure_thr, c->cflags, c->H,
                           c->caux, c->cstat, s);
  });
  timed(c, T_CL_LISTS, [&] {
    launch_closure_lists(c->cflags, c->cvalid, g, p, c->clists, c->ccounts, s);
  });
  // the refreshed cells' new g, with its row sums (closure cells keep g and their sums)
  timed(c, T_CL_GHAT, [&] {
    launch_closure_ghat(G, c->prim, g, dt, eps, c->ms, c->clists + 2 * nc, c->ccounts + 2,
                        c->blocks_g, s, c->rmom);
  });
  timed(c, T_MICRO_X, [&] {
    launch_micro_x_list<double>(G, Gs, c->prim, g, p, dt, c->ms, c->clists, c->ccounts,
                                c->blocks_x, s, c->rmom, c->etab);
  });
  timed(c, T_MICRO_Y, [&] {
    launch_micro_y_list<double>(Gs, G, c->H, c->prim, g, p, dt, eps, c->ms, c->err,
                                c->clists + nc, c->ccounts + 1, c->blocks_y, s, c->rmom,
                                c->etab);
  });
  if (c->n_wall > 0)
    timed(c, T_MICRO_YW, [&] {
      launch_micro_y_wall<double>(Gs, G, c->H, c->prim, c->wall_cells, c->n_wall, g, p, dt, eps,
                                  c->ms, c->err, s, c->rmom);
    });
  timed(c, T_MACRO_X1, [&] { launch_macro_x1(c->Q, c->mb, g, p, dt, eps, c->err, s); });
  timed(c, T_MACRO_X2, [&] { launch_macro_x2(c->H, c->mb, g, p, dt, c->err, s); });
  timed(c, T_MACRO_Y, [&] { launch_macro_y(c->H, c->mb, c->Q, g, p, dt, eps, c->err, s); });
  c->closure_steps += 1;
}

// A step with the closure set: an evaluation (hybrid) step every cl_period steps, whose closure
// count (read back once, the one wait of the evaluation) decides whether the following
// cl_period - 1 steps are hybrid or plain; a plain step after hybrid ones first resets the g of
// the closure cells to Ghat(Q^n) (cstale).  The choice depends only on the computed counts, so
// a run is reproducible.
mm_status enqueue_closure_step(mm_ctx* c, double dt, double eps) {
  if (c->cl_left > 0) {
    --c->cl_left;
    if (c->cl_plain) {
      enqueue_plain<double>(c, dt, eps);
      ++c->fallback_steps;
    } else {
      enqueue_hybrid(c, dt, eps);
    }
    return MM_OK;
  }
  enqueue_hybrid(c, dt, eps);
  if (c->cl_period <= 1) return MM_OK;
  if (!c->cl_host) {
    cudaError_t e = cudaMallocHost((void**)&c->cl_host, sizeof(unsigned long long));
    if (e != cudaSuccess) return cuda_fail(c, e, "closure count buffer");
  }
  cudaError_t e = cudaMemcpyAsync(c->cl_host, c->cstat, sizeof(unsigned long long),
                                  cudaMemcpyDeviceToHost, c->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
  if (e != cudaSuccess) return cuda_fail(c, e, "closure count");
  const unsigned long long now = *c->cl_host;
  const double count = (double)(now - c->cl_seen);
  c->cl_seen = now;
  c->cl_plain = count < c->cl_min_frac * (double)c->ncell;
  if (c->cl_plain) c->cstale = true;
  c->cl_left = c->cl_period - 1;
  return MM_OK;
}

mm_status enqueue_step(mm_ctx* c, double dt, double eps) {
  if (c->fp32) enqueue_plain<float>(c, dt, eps);
  else if (c->mlp) return enqueue_closure_step(c, dt, eps);
  else enqueue_plain<double>(c, dt, eps);
  return MM_OK;
}

constexpr int kHostChunks = 16;  // row chunks of g in mm_step_host

// One plain FP64 step whose g^n arrives from host memory while the micro sweeps run.  Three
// streams: the copy stream brings Q, then g in row chunks; the x stream sweeps each chunk once
// its rows have arrived; the context stream computes the per-cell fields, then sweeps each chunk
// in y once the x sweeps of it and of its neighbour chunks are done (with periodic y the first
// chunk's lower neighbour is the last chunk), then the walls and the macro update.  x sweeps of
// later chunks run beside y sweeps of earlier ones.  Every cell is computed by the same kernels
// as in enqueue_plain, so the result is the same bit for bit.
mm_status enqueue_step_from_host(mm_ctx* c, const double* Q_host, const double* G_host,
                                 double dt, double eps) {
  const KGrid& g = c->kg;
  const KParams& p = c->kp;
  cudaStream_t s = c->stream;
  cudaError_t e = cudaSuccess;
  if (!c->cstream) e = cudaStreamCreateWithFlags(&c->cstream, cudaStreamNonBlocking);
  if (e == cudaSuccess && !c->xstream)
    e = cudaStreamCreateWithFlags(&c->xstream, cudaStreamNonBlocking);
  if (e == cudaSuccess && !c->ystream)
    e = cudaStreamCreateWithFlags(&c->ystream, cudaStreamNonBlocking);
  // row chunks of about ny / kHostChunks rows, the first two a quarter and a half of that: the
  // sweeps start as soon as the first small chunk has arrived
  std::vector<int> bounds{0};
  {
    const int full = std::max(1, (g.ny + kHostChunks - 1) / kHostChunks);
    int rows = std::max(1, full / 4);
    while (bounds.back() < g.ny) {
      bounds.push_back(std::min(g.ny, bounds.back() + rows));
      rows = std::min(full, 2 * rows);
    }
  }
  const int nchunk = (int)bounds.size() - 1;
  // events: [0, n) chunk copied, [n, 2n) chunk x-swept, 2n entry, 2n+1 Q copied, 2n+2 fields,
  // 2n+3 the y sweeps of the second stream done
  const int nev = 2 * nchunk + 4;
  while (e == cudaSuccess && (int)c->chunk_events.size() < nev) {
    cudaEvent_t ev;
    e = cudaEventCreateWithFlags(&ev, cudaEventDisableTiming);
    if (e == cudaSuccess) c->chunk_events.push_back(ev);
  }
  if (e != cudaSuccess) return cuda_fail(c, e, "copy streams");
  cudaEvent_t* copied = c->chunk_events.data();
  cudaEvent_t* xswept = copied + nchunk;
  cudaEvent_t entry = copied[2 * nchunk], qin = copied[2 * nchunk + 1],
              fields = copied[2 * nchunk + 2], ydone = copied[2 * nchunk + 3];
  double* G = static_cast<double*>(c->G);
  double* Gs = static_cast<double*>(c->Gs);
  const size_t row = (size_t)g.nx * g.nv1 * g.nv2;  // doubles of g per row of cells
  auto row0 = [&](int r) { return bounds[r]; };
  // the copies may overwrite Q and g only after the work already queued on the context stream;
  // host-to-device copies are served in issue order, so Q (which the per-cell fields need
  // first) goes ahead of the chunks of g
  e = cudaEventRecord(entry, s);
  if (e == cudaSuccess) e = cudaStreamWaitEvent(c->cstream, entry, 0);
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(c->Q, Q_host, 6 * c->ncell * sizeof(double), cudaMemcpyHostToDevice,
                        c->cstream);
  if (e == cudaSuccess) e = cudaEventRecord(qin, c->cstream);
  for (int r = 0; r < nchunk && e == cudaSuccess; ++r) {
    const size_t off = row * row0(r), n = row * (row0(r + 1) - row0(r));
    e = cudaMemcpyAsync(G + off, G_host + off, n * sizeof(double), cudaMemcpyHostToDevice,
                        c->cstream);
    if (e == cudaSuccess) e = cudaEventRecord(copied[r], c->cstream);
  }
  if (e == cudaSuccess) e = cudaStreamWaitEvent(s, qin, 0);
  if (e == cudaSuccess && c->cvalid) e = cudaMemsetAsync(c->cvalid, 1, c->ncell, s);
  if (e != cudaSuccess) return cuda_fail(c, e, "copy state in");
  c->cstale = false;
  c->have_state = true;
  enqueue_prims(c, dt, eps, s);
  cudaEventRecord(fields, s);
  cudaStreamWaitEvent(c->xstream, fields, 0);
  for (int r = 0; r < nchunk; ++r) {
    cudaStreamWaitEvent(c->xstream, copied[r], 0);
    // the x sweep sums its moments per velocity here (g has just arrived, without row sums);
    // the y sweeps leave the row sums of G^{n+1} for the steps that follow
    const int c0 = row0(r) * g.nx, cn = (row0(r + 1) - row0(r)) * g.nx;
    launch_micro_x<double>(G, Gs, c->prim, g, p, dt, c->ms, c->xstream, c0, cn, c->etab);
    cudaEventRecord(xswept[r], c->xstream);
  }
  // the y sweeps of consecutive chunks alternate between the context stream and a second
  // stream: they write disjoint rows (of g, H and the row sums) and read only x-swept rows, so
  // one chunk's last wave of CTAs can share the GPU with the next chunk's first
  auto ysweep = [&](int r, int after) {
    cudaStream_t ys = (r & 1) ? c->ystream : s;
    cudaStreamWaitEvent(ys, xswept[after], 0);
    timed_on(c, T_MICRO_Y, ys, [&] {
      launch_micro_y<double>(Gs, G, c->H, c->prim, g, p, dt, eps, c->ms, c->err, ys, nullptr,
                             row0(r) * g.nx, (row0(r + 1) - row0(r)) * g.nx, c->rmom,
                             c->etab);
    });
  };
  // x sweeps complete in chunk order, so waiting for chunk r+1 covers chunks 0..r+1
  const bool pery = p.bc[2] == MM_BC_PERIODIC;
  for (int r = pery && nchunk > 1 ? 1 : 0; r < nchunk; ++r) ysweep(r, std::min(r + 1, nchunk - 1));
  if (pery && nchunk > 1) ysweep(0, nchunk - 1);
  // the second stream's sweeps (the last of them waited for every x sweep) before the rest
  cudaEventRecord(ydone, c->ystream);
  cudaStreamWaitEvent(s, ydone, 0);
  if (c->n_wall > 0)
    timed(c, T_MICRO_YW, [&] {
      launch_micro_y_wall<double>(Gs, G, c->H, c->prim, c->wall_cells, c->n_wall, g, p, dt, eps,
                                  c->ms, c->err, s, c->rmom);
    });
  timed(c, T_MACRO_X1, [&] { launch_macro_x1(c->Q, c->mb, g, p, dt, eps, c->err, s); });
  timed(c, T_MACRO_X2, [&] { launch_macro_x2(c->H, c->mb, g, p, dt, c->err, s); });
  timed(c, T_MACRO_Y, [&] { launch_macro_y(c->H, c->mb, c->Q, g, p, dt, eps, c->err, s); });
  e = cudaGetLastError();
  if (e != cudaSuccess) return cuda_fail(c, e, "kernel launch");
  return MM_OK;
}

// Buffers of the closure, allocated on first use.
mm_status ensure_closure(mm_ctx* c) {
  if (c->caux) return MM_OK;
  const size_t nc = c->ncell;
  cudaError_t e = cudaSuccess;
  auto alloc = [&](void** ptr, size_t bytes) {
    if (e == cudaSuccess) e = cudaMalloc(ptr, bytes);
  };
  alloc((void**)&c->cX, nc * MM_MLP_IN * sizeof(float));
  alloc((void**)&c->cY, nc * MM_MLP_OUT * sizeof(float));
  alloc((void**)&c->caux, 5 * nc * sizeof(double));
  alloc((void**)&c->cflags, nc);
  alloc((void**)&c->cvalid, nc);
  alloc((void**)&c->clists, 3 * nc * sizeof(int));
  alloc((void**)&c->ccounts, 3 * sizeof(int));
  alloc((void**)&c->cstat, sizeof(unsigned long long));
  if (e == cudaSuccess) e = cudaMemsetAsync(c->cstat, 0, sizeof(unsigned long long), c->stream);
  if (e == cudaSuccess) e = cudaMemsetAsync(c->cflags, 0, nc, c->stream);
  if (e == cudaSuccess) e = cudaMemsetAsync(c->cvalid, 1, nc, c->stream);
  if (e != cudaSuccess) {
    cudaFree(c->cX); cudaFree(c->cY); cudaFree(c->caux); cudaFree(c->cflags); cudaFree(c->cvalid);
    cudaFree(c->clists); cudaFree(c->ccounts); cudaFree(c->cstat);
    c->cX = c->cY = nullptr; c->caux = nullptr; c->cflags = c->cvalid = nullptr;
    c->clists = c->ccounts = nullptr;
    c->cstat = nullptr;
    return e == cudaErrorMemoryAllocation ? fail(c, MM_ERR_OOM, "closure buffers")
                                          : cuda_fail(c, e, "closure buffers");
  }
  c->blocks_x = micro_list_blocks(c->ms, false);
  c->blocks_y = micro_list_blocks(c->ms, true);
  c->blocks_g = closure_ghat_blocks(c->ms);
  return MM_OK;
}

// Copy an FP64 array of n elements into the context's G (FP64 or FP32), staging through Gs.
mm_status copy_g_in(mm_ctx* c, const double* src, cudaMemcpyKind kind) {
  const size_t n = c->nphase;
  if (!c->fp32) {
    cudaError_t e = cudaMemcpyAsync(c->G, src, n * sizeof(double), kind, c->stream);
    return e == cudaSuccess ? MM_OK : cuda_fail(c, e, "copy G in");
  }
  // FP32 storage: stage chunks of doubles through the scratch buffer Gs (n floats = n/2 doubles)
  const size_t chunk = n / 2 > 0 ? n / 2 : 1;
  double* stage = static_cast<double*>(c->Gs);
  for (size_t off = 0; off < n; off += chunk) {
    const size_t m = off + chunk <= n ? chunk : n - off;
    cudaError_t e = cudaMemcpyAsync(stage, src + off, m * sizeof(double), kind, c->stream);
    if (e != cudaSuccess) return cuda_fail(c, e, "copy G in");
    launch_convert_f64_to_f32(stage, static_cast<float*>(c->G) + off, m, c->stream);
    if (kind == cudaMemcpyHostToDevice) {
      e = cudaStreamSynchronize(c->stream);
      if (e != cudaSuccess) return cuda_fail(c, e, "copy G in");
    }
  }
  return MM_OK;
}

mm_status copy_g_out(mm_ctx* c, double* dst) {
  const size_t n = c->nphase;
  if (!c->fp32) {
    cudaError_t e = cudaMemcpyAsync(dst, c->G, n * sizeof(double), cudaMemcpyDeviceToHost, c->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
    return e == cudaSuccess ? MM_OK : cuda_fail(c, e, "copy G out");
  }
  const size_t chunk = n / 2 > 0 ? n / 2 : 1;
  double* stage = static_cast<double*>(c->Gs);
  for (size_t off = 0; off < n; off += chunk) {
    const size_t m = off + chunk <= n ? chunk : n - off;
    launch_convert_f32_to_f64(static_cast<const float*>(c->G) + off, stage, m, c->stream);
    cudaError_t e = cudaMemcpyAsync(dst + off, stage, m * sizeof(double), cudaMemcpyDeviceToHost, c->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
    if (e != cudaSuccess) return cuda_fail(c, e, "copy G out");
  }
  return MM_OK;
}


// Everything of a context but its device buffers: grid and parameters in kernel form, launch
// shape, sizes and the diffuse-wall cell list.
void init_shape(mm_ctx* c, const mm_grid* grid, const mm_params* params, std::vector<int>& walls) {
  c->grid = *grid;
  c->params = *params;
  c->fp32 = params->precision == MM_PREC_G_FP32;
  c->ncell = (size_t)grid->nx * grid->ny;
  c->nphase = c->ncell * grid->nv1 * grid->nv2;
  KGrid& kg = c->kg;
  kg.nx = grid->nx;
  kg.ny = grid->ny;
  kg.nv1 = grid->nv1;
  kg.nv2 = grid->nv2;
  kg.dx = (grid->x1 - grid->x0) / grid->nx;
  kg.dy = (grid->y1 - grid->y0) / grid->ny;
  kg.idx = 1.0 / kg.dx;
  kg.idy = 1.0 / kg.dy;
  kg.v1min = grid->v1min;
  kg.v2min = grid->v2min;
  kg.dv1 = (grid->v1max - grid->v1min) / grid->nv1;
  kg.dv2 = (grid->v2max - grid->v2min) / grid->nv2;
  KParams& kp = c->kp;
  kp.nu = params->nu;
  kp.tau0 = params->tau0;
  kp.tau_model = params->tau_model;
  for (int s = 0; s < 4; ++s) {
    kp.bc[s] = params->bc[s];
    kp.wall_T[s] = params->wall_T[s];
    kp.wall_U[s] = params->wall_U[s];
  }
  kp.keep_es = params->wall_keep_es_term ? 1 : 0;
  c->ms = micro_shape(grid->nv1, grid->nv2);
  walls.clear();
  for (int j = 0; j < grid->ny; ++j)
    for (int i = 0; i < grid->nx; ++i)
      if ((i == 0 && kp.bc[0] == MM_BC_DIFFUSE) || (i == grid->nx - 1 && kp.bc[1] == MM_BC_DIFFUSE) ||
          (j == 0 && kp.bc[2] == MM_BC_DIFFUSE) || (j == grid->ny - 1 && kp.bc[3] == MM_BC_DIFFUSE))
        walls.push_back(j * grid->nx + i);
  c->n_wall = (int)walls.size();
}

// Every device buffer of a context except Q and G, in a fixed order: mm_create allocates them,
// mm_create_borrowed carves them from the caller's scratch and mm_scratch_bytes adds up their
// sizes, so the three agree by construction.
template <typename F>
void scratch_plan(mm_ctx* c, F&& take) {
  const size_t gsz = c->fp32 ? sizeof(float) : sizeof(double);
  const KParams& kp = c->kp;
  const bool any_diffuse = kp.bc[0] == MM_BC_DIFFUSE || kp.bc[1] == MM_BC_DIFFUSE ||
                           kp.bc[2] == MM_BC_DIFFUSE || kp.bc[3] == MM_BC_DIFFUSE;
  take(&c->Gs, std::max<size_t>(c->nphase * gsz, 16));  // also stages FP64 chunks
  take((void**)&c->macro, macro_doubles(c->kg.nx, c->kg.ny) * sizeof(double));
  take((void**)&c->H, 4 * c->ncell * sizeof(double));
  if (c->fp32) take((void**)&c->Hf, 8 * c->ncell * sizeof(float));
  if (c->fp32 && any_diffuse) take(&c->Gexp, c->nphase * gsz);
  take((void**)&c->prim, NPRIM * c->ncell * sizeof(double));
  if (c->fp32) take((void**)&c->primf, NPRIMF * c->ncell * sizeof(float));
  // row sums for the FP64 sweeps that run one warp per cell with one row per pass
  if (!c->fp32 && c->ms.R == 1 && c->ms.threads == 32)
    take((void**)&c->rmom, 3 * c->ncell * c->kg.nv1 * sizeof(double));
  // the Maxwellian factors e1, e2 of every cell, formed by the x sweep, read by the y sweep
  if (!c->fp32) take((void**)&c->etab, c->ncell * (c->kg.nv1 + c->kg.nv2) * sizeof(double));
  take((void**)&c->err, sizeof(int));
  if (c->n_wall > 0) take((void**)&c->wall_cells, (size_t)c->n_wall * sizeof(int));
}

constexpr size_t kCarveAlign = 256;

size_t carve_round(size_t bytes) { return (bytes + kCarveAlign - 1) / kCarveAlign * kCarveAlign; }

struct Borrowed {
  double* Q;
  void* G;
  char* scratch;
  size_t bytes;
};

mm_status create_ctx(const mm_grid* grid, const mm_params* params, void* cuda_stream,
                     const Borrowed* bw, mm_ctx** out) {
  mm_ctx* c = new mm_ctx();
  c->stream = static_cast<cudaStream_t>(cuda_stream);
  cudaGetDevice(&c->device);
  std::vector<int> walls;
  init_shape(c, grid, params, walls);
  const size_t gsz = c->fp32 ? sizeof(float) : sizeof(double);
  cudaError_t e = cudaSuccess;
  if (!bw) {
    auto alloc = [&](void** ptr, size_t bytes) {
      if (e == cudaSuccess) e = cudaMalloc(ptr, bytes > 0 ? bytes : 1);
    };
    alloc(&c->G, c->nphase * gsz);
    alloc((void**)&c->Q, 6 * c->ncell * sizeof(double));
    scratch_plan(c, alloc);
  } else {
    c->borrowed = true;
    c->G = c->user_G = bw->G;
    c->Q = bw->Q;
    size_t off = 0;
    scratch_plan(c, [&](void** ptr, size_t bytes) {
      *ptr = bw->scratch + off;
      off += carve_round(bytes);
    });
  }
  if (e != cudaSuccess) {
    mm_destroy(c);
    cudaGetLastError();
    return e == cudaErrorMemoryAllocation ? MM_ERR_OOM : MM_ERR_CUDA;
  }
  c->mb = carve_macro(c->macro, grid->nx, grid->ny);
  if (c->fp32) c->nseg = fused_segments_f32(c->kg, c->ms);
  if (c->n_wall > 0)
    e = cudaMemcpyAsync(c->wall_cells, walls.data(), walls.size() * sizeof(int),
                        cudaMemcpyHostToDevice, c->stream);
  if (e == cudaSuccess) e = cudaMemsetAsync(c->err, 0, sizeof(int), c->stream);
  if (e == cudaSuccess) e = cudaMemsetAsync(c->H, 0, 4 * c->ncell * sizeof(double), c->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
  if (e != cudaSuccess) {
    mm_destroy(c);
    return MM_ERR_CUDA;
  }
  *out = c;
  return MM_OK;
}

// g from G_src (or zero), then the closure validity and the row sums: the tail of the setters
mm_status set_g(mm_ctx* c, const double* G_src, cudaMemcpyKind kind) {
  cudaError_t e = cudaSuccess;
  if (G_src) {
    mm_status s = copy_g_in(c, G_src, kind);
    if (s != MM_OK) return s;
  } else {
    e = cudaMemsetAsync(c->G, 0, c->nphase * (c->fp32 ? sizeof(float) : sizeof(double)), c->stream);
    if (e != cudaSuccess) return cuda_fail(c, e, "zero G");
  }
  if (c->cvalid) {
    e = cudaMemsetAsync(c->cvalid, 1, c->ncell, c->stream);
    if (e != cudaSuccess) return cuda_fail(c, e, "reset closure validity");
    c->cstale = false;
  }
  if (c->rmom) launch_row_sums(static_cast<const double*>(c->G), c->rmom, c->kg, c->stream);
  return MM_OK;
}

}  // namespace

extern "C" {

mm_status mm_create(const mm_grid* grid, const mm_params* params, void* cuda_stream,
                    mm_ctx** out) {
  if (!out) return MM_ERR_INVALID_ARG;
  *out = nullptr;
  if (!validate(grid, params).empty()) return MM_ERR_INVALID_ARG;
  return create_ctx(grid, params, cuda_stream, nullptr, out);
}

// G and Q plus every other buffer of the plan (each counted rounded up to the carve alignment)
size_t mm_device_bytes(const mm_grid* grid, const mm_params* params) {
  if (!validate(grid, params).empty()) return 0;
  const size_t nc = (size_t)grid->nx * grid->ny;
  const size_t gs = params->precision == MM_PREC_G_FP32 ? sizeof(float) : sizeof(double);
  return nc * grid->nv1 * grid->nv2 * gs + 6 * nc * sizeof(double) +
         mm_scratch_bytes(grid, params);
}

size_t mm_scratch_bytes(const mm_grid* grid, const mm_params* params) {
  if (!validate(grid, params).empty()) return 0;
  mm_ctx c;
  std::vector<int> walls;
  init_shape(&c, grid, params, walls);
  size_t total = 0;
  scratch_plan(&c, [&](void**, size_t bytes) { total += carve_round(bytes); });
  return total;
}

mm_status mm_create_borrowed(const mm_grid* grid, const mm_params* params, void* cuda_stream,
                             double* Q_dev, void* G_dev, void* scratch_dev, size_t scratch_bytes,
                             mm_ctx** out) {
  if (!out) return MM_ERR_INVALID_ARG;
  *out = nullptr;
  if (!validate(grid, params).empty()) return MM_ERR_INVALID_ARG;
  if (!Q_dev || !G_dev || !scratch_dev) return MM_ERR_INVALID_ARG;
  if ((uintptr_t)Q_dev % 16 != 0 || (uintptr_t)G_dev % kCarveAlign != 0 ||
      (uintptr_t)scratch_dev % kCarveAlign != 0)
    return MM_ERR_INVALID_ARG;
  if (scratch_bytes < mm_scratch_bytes(grid, params)) return MM_ERR_INVALID_ARG;
  const Borrowed bw{Q_dev, G_dev, static_cast<char*>(scratch_dev), scratch_bytes};
  return create_ctx(grid, params, cuda_stream, &bw, out);
}

mm_status mm_set_state(mm_ctx* c, const double* Q_host, const double* G_host) {
  if (!c) return MM_ERR_INVALID_ARG;
  if (!Q_host) return fail(c, MM_ERR_INVALID_ARG, "Q_host is NULL");
  cudaError_t e = cudaMemcpyAsync(c->Q, Q_host, 6 * c->ncell * sizeof(double),
                                  cudaMemcpyHostToDevice, c->stream);
  if (e != cudaSuccess) return cuda_fail(c, e, "copy Q in");
  mm_status st = set_g(c, G_host, cudaMemcpyHostToDevice);
  if (st != MM_OK) return st;
  e = cudaStreamSynchronize(c->stream);
  if (e != cudaSuccess) return cuda_fail(c, e, "set state");
  c->have_state = true;
  return MM_OK;
}

mm_status mm_set_state_prim(mm_ctx* c, const double* rho, const double* u1, const double* u2,
                            const double* T) {
  if (!c) return MM_ERR_INVALID_ARG;
  if (!rho || !u1 || !u2 || !T) return fail(c, MM_ERR_INVALID_ARG, "rho, u1, u2 and T are required");
  for (size_t i = 0; i < c->ncell; ++i)
    if (!(rho[i] > 0.0) || !(T[i] > 0.0) || !std::isfinite(rho[i]) || !std::isfinite(T[i]) ||
        !std::isfinite(u1[i]) || !std::isfinite(u2[i]))
      return fail(c, MM_ERR_INVALID_ARG, "rho and T must be positive and finite, u finite");
  // the four fields go through the per-cell coefficient buffer, which the next step rewrites
  const double* f[4] = {rho, u1, u2, T};
  cudaError_t e = cudaSuccess;
  for (int m = 0; m < 4 && e == cudaSuccess; ++m)
    e = cudaMemcpyAsync(c->prim + m * c->ncell, f[m], c->ncell * sizeof(double),
                        cudaMemcpyHostToDevice, c->stream);
  if (e != cudaSuccess) return cuda_fail(c, e, "copy primitive fields in");
  launch_q_from_prim(c->prim, c->Q, (int)c->ncell, c->stream);
  mm_status st = set_g(c, nullptr, cudaMemcpyHostToDevice);  // g = 0
  if (st != MM_OK) return st;
  e = cudaStreamSynchronize(c->stream);
  if (e != cudaSuccess) return cuda_fail(c, e, "set state from primitive fields");
  c->have_state = true;
  return MM_OK;
}

mm_status mm_set_state_device(mm_ctx* c, const double* Q_dev, const double* G_dev) {
  if (!c) return MM_ERR_INVALID_ARG;
  if (!Q_dev) return fail(c, MM_ERR_INVALID_ARG, "Q_dev is NULL");
  cudaError_t e = cudaMemcpyAsync(c->Q, Q_dev, 6 * c->ncell * sizeof(double),
                                  cudaMemcpyDeviceToDevice, c->stream);
  if (e != cudaSuccess) return cuda_fail(c, e, "copy Q in");
  mm_status st = set_g(c, G_dev, cudaMemcpyDeviceToDevice);
  if (st != MM_OK) return st;
  c->have_state = true;
  return MM_OK;
}

mm_status mm_g_region_changed(mm_ctx* c, int i0, int i1, int j0, int j1) {
  if (!c) return MM_ERR_INVALID_ARG;
  if (i0 < 0 || j0 < 0 || i1 > c->grid.nx || j1 > c->grid.ny || i0 > i1 || j0 > j1)
    return fail(c, MM_ERR_INVALID_ARG, "region outside the grid");
  if (c->rmom)
    launch_row_sums_rect(static_cast<const double*>(c->G), c->rmom, c->kg, i0, i1, j0, j1,
                         c->stream);
  cudaError_t e = cudaGetLastError();
  return e == cudaSuccess ? MM_OK : cuda_fail(c, e, "row sums of a region");
}

mm_status mm_step(mm_ctx* c, double dt, double eps, int nsteps) {
  if (!c) return MM_ERR_INVALID_ARG;
  if (!(dt > 0.0) || !std::isfinite(dt)) return fail(c, MM_ERR_INVALID_ARG, "dt must be > 0");
  if (!(eps > 0.0) || !std::isfinite(eps)) return fail(c, MM_ERR_INVALID_ARG, "eps must be > 0");
  if (nsteps < 0) return fail(c, MM_ERR_INVALID_ARG, "nsteps must be >= 0");
  if (!c->have_state) return fail(c, MM_ERR_STATE, "mm_step before mm_set_state");
  for (int n = 0; n < nsteps; ++n) {
    mm_status st = enqueue_step(c, dt, eps);
    if (st != MM_OK) return st;
  }
  if (c->borrowed && c->G != c->user_G) {
    // FP32 g ping-pongs between G and the scratch copy: leave the state in the caller's buffer
    cudaMemcpyAsync(c->user_G, c->G, c->nphase * sizeof(float), cudaMemcpyDeviceToDevice,
                    c->stream);
    std::swap(c->G, c->Gs);
  }
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return cuda_fail(c, e, "kernel launch");
  return MM_OK;
}

mm_status mm_sync(mm_ctx* c) {
  if (!c) return MM_ERR_INVALID_ARG;
  cudaError_t e = cudaStreamSynchronize(c->stream);
  if (e != cudaSuccess) return cuda_fail(c, e, "stream synchronize");
  return check_device_errors(c);
}

mm_status mm_get_moments(mm_ctx* c, double* Q_host, double* H_host) {
  if (!c) return MM_ERR_INVALID_ARG;
  if (!Q_host) return fail(c, MM_ERR_INVALID_ARG, "Q_host is NULL");
  cudaError_t e = cudaMemcpyAsync(Q_host, c->Q, 6 * c->ncell * sizeof(double),
                                  cudaMemcpyDeviceToHost, c->stream);
  if (e == cudaSuccess && H_host)
    e = cudaMemcpyAsync(H_host, c->H, 4 * c->ncell * sizeof(double), cudaMemcpyDeviceToHost,
                        c->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
  if (e != cudaSuccess) return cuda_fail(c, e, "copy moments out");
  return check_device_errors(c);
}

mm_status mm_step_host(mm_ctx* c, const double* Q_host, const double* G_host, double dt,
                       double eps, double* Q_out, double* H_out) {
  if (!c) return MM_ERR_INVALID_ARG;
  if (!Q_host || !G_host || !Q_out)
    return fail(c, MM_ERR_INVALID_ARG, "Q_host, G_host and Q_out are required");
  if (!(dt > 0.0) || !std::isfinite(dt)) return fail(c, MM_ERR_INVALID_ARG, "dt must be > 0");
  if (!(eps > 0.0) || !std::isfinite(eps)) return fail(c, MM_ERR_INVALID_ARG, "eps must be > 0");
  if (c->fp32 || c->mlp || c->mms) {  // not pipelined: the same three calls in sequence
    mm_status st = mm_set_state(c, Q_host, G_host);
    if (st == MM_OK) st = mm_step(c, dt, eps, 1);
    if (st == MM_OK) st = mm_get_moments(c, Q_out, H_out);
    return st;
  }
  mm_status st = enqueue_step_from_host(c, Q_host, G_host, dt, eps);
  if (st != MM_OK) return st;
  return mm_get_moments(c, Q_out, H_out);
}

mm_status mm_get_moments_device(mm_ctx* c, double* Q_dev, double* H_dev) {
  if (!c) return MM_ERR_INVALID_ARG;
  if (!Q_dev) return fail(c, MM_ERR_INVALID_ARG, "Q_dev is NULL");
  cudaError_t e = cudaMemcpyAsync(Q_dev, c->Q, 6 * c->ncell * sizeof(double),
                                  cudaMemcpyDeviceToDevice, c->stream);
  if (e == cudaSuccess && H_dev)
    e = cudaMemcpyAsync(H_dev, c->H, 4 * c->ncell * sizeof(double), cudaMemcpyDeviceToDevice,
                        c->stream);
  if (e != cudaSuccess) return cuda_fail(c, e, "copy moments out");
  return MM_OK;
}

mm_status mm_get_g(mm_ctx* c, double* G_host) {
  if (!c) return MM_ERR_INVALID_ARG;
  if (!G_host) return fail(c, MM_ERR_INVALID_ARG, "G_host is NULL");
  mm_status s = copy_g_out(c, G_host);
  if (s != MM_OK) return s;
  return check_device_errors(c);
}

double mm_dt_for_cfl(const mm_grid* g, double cfl, double t_final, int form, int* nsteps_out) {
  if (!g || g->nx < 1 || g->ny < 1 || !(cfl > 0.0) || !(g->x1 > g->x0) || !(g->y1 > g->y0))
    return -1.0;
  const double dx = (g->x1 - g->x0) / g->nx;
  const double dy = (g->y1 - g->y0) / g->ny;
  const double V1 = std::fmax(std::fabs(g->v1min), std::fabs(g->v1max));
  const double V2 = std::fmax(std::fabs(g->v2min), std::fabs(g->v2max));
  if (!(V1 > 0.0) || (g->ny > 1 && !(V2 > 0.0))) return -1.0;
  double dt;
  if (g->ny == 1) dt = cfl * dx / V1;
  else if (form == MM_CFL_MIN) dt = cfl * std::fmin(dx / V1, dy / V2);
  else dt = cfl / (V1 / dx + V2 / dy);
  int n = 0;
  if (t_final > 0.0) {
    n = (int)std::ceil(t_final / dt * (1.0 - 1e-12));
    if (n < 1) n = 1;
    dt = t_final / n;
  }
  if (nsteps_out) *nsteps_out = n;
  return dt;
}

// Velocity tables and source buffers of the manufactured-solution harness, on first use.
mm_status ensure_mms(mm_ctx* c) {
  if (c->mms_phi) return MM_OK;
  const size_t nv = (size_t)c->grid.nv1 * c->grid.nv2;
  cudaError_t e = cudaMalloc(&c->mms_phi, nv * sizeof(double));
  if (e == cudaSuccess) e = cudaMalloc(&c->mms_gam, nv * sizeof(double));
  if (e == cudaSuccess) e = cudaMalloc(&c->mms_src_g, c->nphase * sizeof(double));
  if (e == cudaSuccess) e = cudaMalloc(&c->mms_src_q, 6 * c->ncell * sizeof(double));
  if (e != cudaSuccess) {
    cudaFree(c->mms_phi); cudaFree(c->mms_gam); cudaFree(c->mms_src_g); cudaFree(c->mms_src_q);
    c->mms_phi = c->mms_gam = c->mms_src_g = c->mms_src_q = nullptr;
    return e == cudaErrorMemoryAllocation ? fail(c, MM_ERR_OOM, "manufactured-solution buffers")
                                          : cuda_fail(c, e, "manufactured-solution buffers");
  }
  launch_mms_tables(c->mms_phi, c->mms_gam, c->kg, c->kp, c->stream);
  return MM_OK;
}

mm_status mms_check(mm_ctx* c) {
  if (c->fp32) return fail(c, MM_ERR_INVALID_ARG, "the manufactured solution needs an FP64 context");
  for (int s = 0; s < 4; ++s)
    if (c->kp.bc[s] != MM_BC_PERIODIC)
      return fail(c, MM_ERR_INVALID_ARG, "the manufactured solution is doubly periodic");
  return MM_OK;
}

mm_status mm_mms_enable(mm_ctx* c, int enable, double t0) {
  if (!c) return MM_ERR_INVALID_ARG;
  if (!enable) {
    c->mms = false;
    return MM_OK;
  }
  mm_status st = mms_check(c);
  if (st != MM_OK) return st;
  if (c->mlp) return fail(c, MM_ERR_STATE, "switch the closure off before the manufactured source");
  if (!std::isfinite(t0)) return fail(c, MM_ERR_INVALID_ARG, "t0 must be finite");
  st = ensure_mms(c);
  if (st != MM_OK) return st;
  c->mms = true;
  c->mms_t = t0;
  return MM_OK;
}

mm_status mm_mms_set_exact(mm_ctx* c, double t, double eps) {
  if (!c) return MM_ERR_INVALID_ARG;
  mm_status st = mms_check(c);
  if (st != MM_OK) return st;
  if (!(eps > 0.0) || !std::isfinite(t)) return fail(c, MM_ERR_INVALID_ARG, "bad t or eps");
  st = ensure_mms(c);
  if (st != MM_OK) return st;
  launch_mms_exact(c->Q, static_cast<double*>(c->G), c->mms_phi, c->kg, c->kp, t, eps,
                   c->grid.x0, c->grid.y0, c->stream);
  if (c->rmom) launch_row_sums(static_cast<const double*>(c->G), c->rmom, c->kg, c->stream);
  if (c->cvalid) cudaMemsetAsync(c->cvalid, 1, c->ncell, c->stream);
  c->cstale = false;
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return cuda_fail(c, e, "manufactured initial state");
  c->have_state = true;
  return MM_OK;
}

mm_status mm_mms_error(mm_ctx* c, double t, double eps, double* macro_err, double* micro_err) {
  if (!c) return MM_ERR_INVALID_ARG;
  mm_status st = mms_check(c);
  if (st != MM_OK) return st;
  if (!c->have_state) return fail(c, MM_ERR_STATE, "no state set");
  st = ensure_mms(c);
  if (st != MM_OK) return st;
  double* sums = nullptr;
  cudaError_t e = cudaMalloc(&sums, 4 * c->ncell * sizeof(double));
  if (e != cudaSuccess) return cuda_fail(c, e, "error sums");
  launch_mms_errors(c->Q, static_cast<const double*>(c->G), c->mms_phi, sums, c->kg, c->kp, t,
                    eps, c->grid.x0, c->grid.y0, c->stream);
  std::vector<double> h(4 * c->ncell);
  e = cudaMemcpyAsync(h.data(), sums, h.size() * sizeof(double), cudaMemcpyDeviceToHost, c->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
  cudaFree(sums);
  if (e != cudaSuccess) return cuda_fail(c, e, "error sums");
  double a[4] = {0, 0, 0, 0};
  for (int m = 0; m < 4; ++m)
    for (size_t k = 0; k < c->ncell; ++k) a[m] += h[m * c->ncell + k];
  if (macro_err) *macro_err = std::sqrt(a[0] / a[1]);
  if (micro_err) *micro_err = std::sqrt(a[2] / a[3]);
  return check_device_errors(c);
}

mm_status mm_set_closure(mm_ctx* c, const mm_mlp* m, double threshold) {
  if (!c) return MM_ERR_INVALID_ARG;
  if (m && c->mms) return fail(c, MM_ERR_STATE, "switch the manufactured source off first");
  if (!m) {
    if (c->mlp) c->cstale = true;  // the next plain step first resets non-current g to Ghat
    c->mlp = nullptr;
    return MM_OK;
  }
  if (c->fp32) return fail(c, MM_ERR_INVALID_ARG, "the closure needs an FP64 context");
  if (!(threshold >= 0.0) || !std::isfinite(threshold))
    return fail(c, MM_ERR_INVALID_ARG, "threshold must be finite and >= 0");
  mm_status st = ensure_closure(c);
  if (st != MM_OK) return st;
  cudaError_t e = cudaMemsetAsync(c->cstat, 0, sizeof(unsigned long long), c->stream);
  if (e != cudaSuccess) return cuda_fail(c, e, "reset closure statistics");
  c->mlp = m;
  c->closure_thr = threshold;
  c->closure_steps = 0;
  c->cstale = false;
  c->cl_left = 0;
  c->cl_plain = false;
  c->cl_seen = 0;
  c->fallback_steps = 0;
  return MM_OK;
}

mm_status mm_set_closure_fallback(mm_ctx* c, double min_fraction, int period) {
  if (!c) return MM_ERR_INVALID_ARG;
  if (!(min_fraction >= 0.0 && min_fraction <= 1.0) || period < 1)
    return fail(c, MM_ERR_INVALID_ARG, "need 0 <= min_fraction <= 1 and period >= 1");
  c->cl_min_frac = min_fraction;
  c->cl_period = period;
  c->cl_left = 0;
  c->cl_plain = false;
  return MM_OK;
}

mm_status mm_closure_steps(mm_ctx* c, long long* hybrid_steps, long long* plain_steps) {
  if (!c) return MM_ERR_INVALID_ARG;
  if (hybrid_steps) *hybrid_steps = c->closure_steps;
  if (plain_steps) *plain_steps = c->fallback_steps;
  return MM_OK;
}

mm_status mm_closure_features(mm_ctx* c, double dt, double eps, float* X_dev, double* aux_dev) {
  if (!c) return MM_ERR_INVALID_ARG;
  if (!X_dev || !aux_dev) return fail(c, MM_ERR_INVALID_ARG, "null output");
  if (!(dt > 0.0) || !(eps > 0.0)) return fail(c, MM_ERR_INVALID_ARG, "dt and eps must be > 0");
  if (!c->have_state) return fail(c, MM_ERR_STATE, "no state set");
  enqueue_prims(c, dt, eps, c->stream);
  launch_closure_features(c->Q, c->prim, c->kg, c->kp, eps, dt, X_dev, aux_dev, c->stream);
  cudaError_t e = cudaGetLastError();
  return e == cudaSuccess ? MM_OK : cuda_fail(c, e, "closure features");
}

mm_status mm_closure_collect(mm_ctx* c, double dt, double eps, float* X_dev, float* Y_dev) {
  if (!c) return MM_ERR_INVALID_ARG;
  if (!X_dev || !Y_dev) return fail(c, MM_ERR_INVALID_ARG, "null output");
  if (!(dt > 0.0) || !std::isfinite(dt) || !(eps > 0.0) || !std::isfinite(eps))
    return fail(c, MM_ERR_INVALID_ARG, "dt and eps must be finite and > 0");
  if (!c->have_state) return fail(c, MM_ERR_STATE, "no state set");
  mm_status st = ensure_closure(c);
  if (st != MM_OK) return st;
  enqueue_prims(c, dt, eps, c->stream);
  launch_closure_features(c->Q, c->prim, c->kg, c->kp, eps, dt, X_dev, c->caux, c->stream);
  if (c->fp32) enqueue_plain<float>(c, dt, eps);
  else enqueue_plain<double>(c, dt, eps);
  launch_closure_targets(c->H, c->caux, Y_dev, c->kg, c->stream);
  cudaError_t e = cudaGetLastError();
  return e == cudaSuccess ? MM_OK : cuda_fail(c, e, "closure collect");
}

mm_status mm_closure_flags(mm_ctx* c, unsigned char* flags_host) {
  if (!c || !flags_host) return MM_ERR_INVALID_ARG;
  if (!c->cflags) return fail(c, MM_ERR_STATE, "no closure step has run");
  cudaError_t e = cudaMemcpyAsync(flags_host, c->cflags, c->ncell, cudaMemcpyDeviceToHost, c->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
  return e == cudaSuccess ? MM_OK : cuda_fail(c, e, "copy closure flags");
}

mm_status mm_closure_stats(mm_ctx* c, long long* closure_cells, long long* cell_steps) {
  if (!c) return MM_ERR_INVALID_ARG;
  unsigned long long h = 0;
  if (c->cstat) {
    cudaError_t e = cudaMemcpyAsync(&h, c->cstat, sizeof h, cudaMemcpyDeviceToHost, c->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
    if (e != cudaSuccess) return cuda_fail(c, e, "closure statistics");
  }
  if (closure_cells) *closure_cells = (long long)h;
  if (cell_steps) *cell_steps = c->closure_steps * (long long)c->ncell;
  return MM_OK;
}

const char* mm_last_error(const mm_ctx* c) { return c ? c->last_error.c_str() : "null context"; }

mm_status mm_set_timing(mm_ctx* c, int enable) {
  if (!c) return MM_ERR_INVALID_ARG;
  cudaError_t e = cudaStreamSynchronize(c->stream);
  if (e != cudaSuccess) return cuda_fail(c, e, "stream synchronize");
  drain_timing(c);
  for (int k = 0; k < kNumKernels; ++k) {
    c->acc_ms[k] = 0.0;
    c->acc_n[k] = 0;
  }
  c->timing = enable != 0;
  return MM_OK;
}

mm_status mm_get_timing(mm_ctx* c, double* ms_out, long long* launches_out) {
  if (!c) return MM_ERR_INVALID_ARG;
  cudaError_t e = cudaStreamSynchronize(c->stream);
  if (e != cudaSuccess) return cuda_fail(c, e, "stream synchronize");
  drain_timing(c);
  for (int k = 0; k < kNumKernels; ++k) {
    if (ms_out) ms_out[k] = c->acc_ms[k];
    if (launches_out) launches_out[k] = c->acc_n[k];
  }
  return MM_OK;
}

int mm_num_kernels(void) { return kNumKernels; }

const char* mm_kernel_name(int idx) {
  return idx >= 0 && idx < kNumKernels ? kKernelNames[idx] : "";
}

void mm_destroy(mm_ctx* c) {
  if (!c) return;
  cudaStreamSynchronize(c->stream);
  if (c->cl_host) cudaFreeHost(c->cl_host);
  destroy_events(c);
  for (cudaEvent_t ev : {c->ev_fork, c->ev_x1})
    if (ev) cudaEventDestroy(ev);
  for (cudaStream_t t : {c->cstream, c->xstream, c->ystream, c->mstream})
    if (t) {
      cudaStreamSynchronize(t);
      cudaStreamDestroy(t);
    }
  for (auto e : c->chunk_events) cudaEventDestroy(e);
  if (c->borrowed) {  // Q, G and the scratch pieces belong to the caller
    c->G = c->Gs = c->Gexp = nullptr;
    c->Q = c->macro = c->H = c->prim = c->rmom = c->etab = nullptr;
    c->Hf = c->primf = nullptr;
    c->err = c->wall_cells = nullptr;
  }
  cudaFree(c->G);
  cudaFree(c->Gs);
  cudaFree(c->Gexp);
  cudaFree(c->Q);
  cudaFree(c->macro);
  cudaFree(c->H);
  cudaFree(c->Hf);
  cudaFree(c->prim);
  cudaFree(c->primf);
  cudaFree(c->rmom);
  cudaFree(c->etab);
  cudaFree(c->err);
  cudaFree(c->wall_cells);
  cudaFree(c->cX);
  cudaFree(c->cY);
  cudaFree(c->caux);
  cudaFree(c->cflags);
  cudaFree(c->cvalid);
  cudaFree(c->clists);
  cudaFree(c->ccounts);
  cudaFree(c->cstat);
  cudaFree(c->mms_phi);
  cudaFree(c->mms_gam);
  cudaFree(c->mms_src_g);
  cudaFree(c->mms_src_q);
  delete c;
}

}  // extern "C"
