// Batched stepping of many independent micro-macro KFVS problems of uneven size and Knudsen
// number (Section 5 of Rossmanith & Sar, arXiv 2509.21832, applied to each problem).
//
// All problems live in one set of concatenated device arrays.  A call of mm_batch_step is ONE
// launch of a persistent kernel for all of its steps: the CTAs take work items from a queue --
// (step, problem, phase, tile of cells) -- in a fixed order, and run on each item the same device
// bodies as the single-problem kernels, with that problem's grid, parameters, dt and eps read
// from a descriptor array in device memory.  The phases of a step are: every cell's (u1, u2, T);
// the per-cell coefficients; the micro x sweep; the micro y sweep with relaxation and heat flux;
// the diffuse-wall cells; and the three macro kernels (collision half step and x half fluxes, x
// transport, y transport and the second half step).  Before running an item a CTA waits until
// the phases it depends on are complete for the same problem (a counter per step, problem and
// phase); waits are bounded (a wait that runs out sets an error bit that mm_batch_sync reports as
// MM_ERR_TIMEOUT and the kernel ends).  Every dependency of an item lies earlier in the queue, and
// a CTA only takes an item while it runs, so every item waited on is held by a running CTA or
// already done: the queue cannot deadlock, whatever the number of resident CTAs.  Data that other
// CTAs of the same launch wrote is read with ordinary (coherent) loads after an acquire of the
// counter (the bodies are compiled here without __restrict__, so no load takes the read-only
// path).  The launch is captured in a CUDA graph (with the reset of its counters) and replayed.
// The tile sizes (cells per item of the phase-space phases and of the per-cell phases) are chosen
// by a small autotuner (timed trial steps on a copy of the batch's own state), cached per process
// by the multiset of problem shapes.  Problems run as one warp per cell with one row per pass keep
// the row sums of g (sum over v2 of v2^j g, j = 0..2, per v1 column) as the single-problem
// contexts do: the y sweep leaves them for the next x sweep.
#define MMK_R
#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <map>
#include <mutex>
#include <string>
#include <vector>

#include "mm_body_macro.cuh"
#include "mm_body_micro.cuh"

using namespace mmk;

namespace {

struct BatchProb {
  KGrid g;
  KParams p;
  double dt, eps, ieps, dtidx, dtidy, hscale;  // ieps = 1/eps, formed on the host
  long long g_off;    // offset of the problem's phase-space block (elements)
  long long mac_off;  // offset of its macro buffers (doubles)
  long long r_off;    // offset of its row sums (3 nv1 doubles per cell; nv1 <= 32 only)
  long long e_off;    // offset of its Maxwellian factors e1, e2 (nv1 + nv2 doubles per cell)
  int c_off;          // first global cell index of the problem
  int w_off;          // first entry of its diffuse-wall cells in the wall list
  int n_wall;
  int R;              // rows per pass of the phase-space mapping for the tuned CTA size
  int rows;           // 1: one warp per cell, R = 1, row sums kept (x sweep from them)
};

__device__ __forceinline__ double* rows_of(double* Rm, const BatchProb& b) {
  return (Rm && b.rows) ? Rm + b.r_off : nullptr;
}

// Phases of one step, in the order of the single-problem step.
enum Phase { PH_UT = 0, PH_PRIMS, PH_X, PH_Y, PH_WALL, PH_MX1, PH_MX2, PH_MY, NPH };

// A work item: cells [begin, end) of problem q in phase ph (for the wall phase, entries
// [begin, end) of the problem's list of diffuse-wall cells).
struct Item {
  int q, ph, begin, end;
};

struct MegaArgs {
  double* G;
  double* Gs;
  double* Q;
  double* H;
  double* prim;
  double* mac;
  double* Rm;
  double* Ee;
  const int* walls;
  const BatchProb* pr;
  const Item* items;     // the items of one step, in queue order
  const int* need;       // [nprob][NPH]: items of each phase of each problem in a step
  unsigned* head;        // next queue position
  unsigned* done;        // [nsteps][nprob][NPH]: completed items
  int* err;
  int nitems, nsteps, nprob;
  long long wait_ns;     // bound of one wait
  int hold_q, hold_ph;   // diagnostic: completions of (hold_q, hold_ph) are not counted (-1: off)
};

__device__ __forceinline__ unsigned long long global_ns() {
  unsigned long long t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}

__device__ __forceinline__ unsigned ld_acquire(const unsigned* p) {
  unsigned v;
  asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
  return v;
}

// Wait (one thread) until *ctr >= need; false when the wait ran out or another CTA's did.
__device__ bool wait_count(const unsigned* ctr, unsigned need, unsigned long long t_end,
                           const int* err) {
  if (need == 0) return true;
  for (;;) {
    if (ld_acquire(ctr) >= need) return true;
    if (*(const volatile int*)err & ERR_WAIT_TIMEOUT) return false;
    if (global_ns() > t_end) return false;
    __nanosleep(128);
  }
}

// Counters an item of phase ph waits on (same problem; prev = the previous step's counters, or
// NULL in the first step of the launch).
__device__ bool wait_deps(const MegaArgs& a, const unsigned* cur, const unsigned* prev, int q,
                          int ph) {
  const int* nd = a.need + q * NPH;
  const unsigned long long t_end = global_ns() + (unsigned long long)a.wait_ns;
  auto w = [&](const unsigned* base, int dep) {
    return wait_count(base + q * NPH + dep, (unsigned)nd[dep], t_end, a.err);
  };
  switch (ph) {
    case PH_UT:
    case PH_MX1:  // Q^n of this step is the previous step's output
      return prev == nullptr || w(prev, PH_MY);
    case PH_PRIMS: return w(cur, PH_UT);
    case PH_X: return w(cur, PH_PRIMS);
    case PH_Y:
    case PH_WALL: return w(cur, PH_X);
    case PH_MX2: return w(cur, PH_MX1) && w(cur, PH_Y) && w(cur, PH_WALL);
    default: return w(cur, PH_MX2);
  }
}

// The whole of nsteps batch steps: persistent CTAs of blockDim.x threads take queue items.
// Compiled for 24 one-warp CTAs per SM (80 registers; the spills fall in the macro and wall
// paths): measured faster than 16 (128 registers) or 20 (96).
__global__ void __launch_bounds__(32, 24) k_batch_steps(MegaArgs a) {
  extern __shared__ double sm[];
  __shared__ int s_item;
  const int t = threadIdx.x, T = blockDim.x;
  const long long total = (long long)a.nitems * a.nsteps;
  for (;;) {
    if (t == 0) {
      int it = -1;
      if (!(*(volatile int*)a.err & ERR_WAIT_TIMEOUT)) {
        const unsigned pos = atomicAdd(a.head, 1u);
        if ((long long)pos < total) {
          it = (int)pos;
          const int step = it / a.nitems;
          const Item w = a.items[it % a.nitems];
          const unsigned* cur = a.done + (size_t)step * a.nprob * NPH;
          const unsigned* prev = step > 0 ? cur - (size_t)a.nprob * NPH : nullptr;
          if (!wait_deps(a, cur, prev, w.q, w.ph)) {
            atomicOr(a.err, ERR_WAIT_TIMEOUT);
            it = -1;
          }
          __threadfence();
        }
      }
      s_item = it;
    }
    __syncthreads();
    const int it = s_item;
    if (it < 0) return;
    const int step = it / a.nitems;
    const Item w = a.items[it % a.nitems];
    const BatchProb& b = a.pr[w.q];
    const int nc = b.g.nx * b.g.ny;
    double* Qp = a.Q + 6 * (size_t)b.c_off;
    double* Hp = a.H + 4 * (size_t)b.c_off;
    double* pp = a.prim + NPRIM * (size_t)b.c_off;
    switch (w.ph) {
      case PH_UT:
        for (int c = w.begin + t; c < w.end; c += T) macro_body::uT_body(Qp, pp, nc, c);
        break;
      case PH_PRIMS:
        for (int c = w.begin + t; c < w.end; c += T)
          macro_body::prims_body<true>(Qp, pp, nullptr, b.g, b.p, b.dt, b.eps, b.ieps, a.err, c);
        break;
      case PH_X:
        for (int c = w.begin; c < w.end; ++c) {
          if (b.rows)
            micro_body::micro_x_rows_body<double>(a.G + b.g_off, a.Gs + b.g_off, pp,
                                                  a.Rm + b.r_off, a.Ee + b.e_off, b.g, b.p,
                                                  b.dtidx, c, sm);
          else
            micro_body::micro_x_body<double>(a.G + b.g_off, a.Gs + b.g_off, pp, b.g, b.p,
                                             b.dtidx, b.R, c, sm, a.Ee + b.e_off);
          __syncthreads();
        }
        break;
      case PH_Y:
        for (int c = w.begin; c < w.end; ++c) {
          micro_body::micro_y_body<double>(a.Gs + b.g_off, a.G + b.g_off, Hp, pp, b.g, b.p,
                                           b.dtidy, b.hscale, b.R, a.err, c, sm, nullptr,
                                           rows_of(a.Rm, b), a.Ee + b.e_off);
          __syncthreads();
        }
        break;
      case PH_WALL:
        for (int k = w.begin; k < w.end; ++k) {
          micro_body::micro_y_wall_body<double>(a.Gs + b.g_off, a.G + b.g_off, Hp, pp, b.g,
                                                b.p, b.dt, b.eps, b.R, a.err,
                                                a.walls[b.w_off + k], sm, rows_of(a.Rm, b));
          __syncthreads();
        }
        break;
      default: {
        const MacroBufs mb = carve_macro(a.mac + b.mac_off, b.g.nx, b.g.ny);
        for (int c = w.begin + t; c < w.end; c += T) {
          if (w.ph == PH_MX1) macro_body::macro_x1_body(Qp, mb, b.g, b.p, b.dt, b.eps, a.err, c);
          else if (w.ph == PH_MX2) macro_body::macro_x2_body(Hp, mb, b.g, b.p, b.dt, a.err, c);
          else macro_body::macro_y_body(Hp, mb, Qp, b.g, b.p, b.dt, b.eps, a.err, c);
        }
      }
    }
    // every thread's writes, then one release of the item's completion at GPU scope
    __threadfence();
    __syncthreads();
    if (t == 0 && !(w.q == a.hold_q && w.ph == a.hold_ph)) {
      __threadfence();
      atomicAdd(a.done + ((size_t)step * a.nprob + w.q) * NPH + w.ph, 1u);
    }
  }
}

struct Tune {
  int threads;     // CTA size (whole warps covering the widest v1 mesh)
  int ctas;        // persistent CTAs
  int tile_micro;  // cells per item of the phase-space phases
  int tile_macro;  // cells per item of the per-cell phases
};

std::mutex g_tune_mutex;
std::map<std::string, Tune> g_tune_cache;

int best_R(int nv1, int nv2, int threads) {
  int best = 1;
  double bu = -1.0;
  for (int R = 1; R * nv1 <= threads && R <= 32; ++R) {
    const int passes = (nv2 + R - 1) / R;
    const double u = (double)(R * nv1) / threads * ((double)nv2 / (R * passes));
    if (u > bu + 1e-9) {
      bu = u;
      best = R;
    }
    if (R >= nv2) break;
  }
  return best;
}

constexpr long long kWaitNs = 2000000000LL;  // bound of one dependency wait: 2 s

}  // namespace

struct mm_batch {
  int nprob = 0;
  std::vector<mm_grid> grids;
  std::vector<mm_params> params;
  std::vector<BatchProb> hp;   // host copy of the descriptors
  std::vector<int> start, wstart;
  cudaStream_t stream = nullptr;
  bool own_stream = false;
  size_t nphase = 0;
  int ncell = 0, nwall = 0;
  int max_nv1 = 0, max_nv2 = 0;
  double* G = nullptr;
  double* Gs = nullptr;
  double* Q = nullptr;
  double* H = nullptr;
  double* prim = nullptr;
  double* mac = nullptr;
  double* Rm = nullptr;  // row sums of every problem with nv1 <= 32
  double* Ee = nullptr;  // e1, e2 of every cell, from the x sweep to the y sweep
  int* walls = nullptr;
  BatchProb* d_prob = nullptr;
  int* err = nullptr;
  // the work queue of one step and its counters
  std::vector<Item> items;
  std::vector<int> need;
  Item* d_items = nullptr;
  int* d_need = nullptr;
  unsigned* d_ctr = nullptr;  // [0]: queue head (padded to 64 entries), then the done counters
  int ctr_steps = 0;          // steps the counters have room for
  Tune tune{32, 152, 1, 32};
  bool use_graph = true;
  cudaGraph_t graph = nullptr;
  cudaGraphExec_t gexec = nullptr;
  int graph_steps = 0;
  long long wait_ns = kWaitNs;
  int hold_q = -1, hold_ph = -1;
  std::vector<double> last_dt, last_eps;
  std::string last_error;
  std::string signature;
};

namespace {

mm_status bfail(mm_batch* b, mm_status s, const std::string& m) {
  if (b) b->last_error = m;
  return s;
}
mm_status bcuda(mm_batch* b, cudaError_t e, const char* what) {
  return bfail(b, MM_ERR_CUDA, std::string(what) + ": " + cudaGetErrorString(e));
}

// Dynamic shared memory of the persistent kernel: the largest need of the three micro bodies.
size_t smem_steps(const mm_batch* b) {
  const size_t x = micro_body::kRed + 4 * (size_t)b->max_nv2;
  const size_t y = micro_body::kRed + micro_body::kYTables * (size_t)b->max_nv2;
  const size_t w = micro_body::wall_smem_doubles(b->max_nv1, b->max_nv2);
  return sizeof(double) * std::max(x, std::max(y, w));
}

// The queue of one step: per group of phases, every problem's items in problem order.  Groups:
// {(u, T), macro x1} {prims} {x sweep} {y sweep, walls} {macro x2} {macro y}.
void build_items(mm_batch* b) {
  b->items.clear();
  b->need.assign((size_t)b->nprob * NPH, 0);
  const int tm = b->tune.tile_micro, tc = b->tune.tile_macro;
  auto add = [&](int q, int ph, int n, int tile) {
    for (int c = 0; c < n; c += tile) {
      b->items.push_back(Item{q, ph, c, std::min(n, c + tile)});
      ++b->need[(size_t)q * NPH + ph];
    }
  };
  const int groups[6][2] = {{PH_UT, PH_MX1}, {PH_PRIMS, -1}, {PH_X, -1}, {PH_Y, PH_WALL},
                            {PH_MX2, -1}, {PH_MY, -1}};
  for (const auto& gr : groups)
    for (int k = 0; k < 2; ++k) {
      const int ph = gr[k];
      if (ph < 0) continue;
      for (int q = 0; q < b->nprob; ++q) {
        const BatchProb& d = b->hp[q];
        const int nc = d.g.nx * d.g.ny;
        if (ph == PH_X || ph == PH_Y) add(q, ph, nc, tm);
        else if (ph == PH_WALL) add(q, ph, d.n_wall, tm);
        else add(q, ph, nc, tc);
      }
    }
}

void drop_graph(mm_batch* b) {
  if (b->gexec) cudaGraphExecDestroy(b->gexec);
  if (b->graph) cudaGraphDestroy(b->graph);
  b->gexec = nullptr;
  b->graph = nullptr;
  b->graph_steps = 0;
}

mm_status upload_items(mm_batch* b) {
  cudaFree(b->d_items);
  cudaFree(b->d_need);
  b->d_items = nullptr;
  b->d_need = nullptr;
  cudaError_t e = cudaMalloc((void**)&b->d_items, sizeof(Item) * std::max<size_t>(1, b->items.size()));
  if (e == cudaSuccess) e = cudaMalloc((void**)&b->d_need, sizeof(int) * b->need.size());
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(b->d_items, b->items.data(), sizeof(Item) * b->items.size(),
                        cudaMemcpyHostToDevice, b->stream);
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(b->d_need, b->need.data(), sizeof(int) * b->need.size(),
                        cudaMemcpyHostToDevice, b->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(b->stream);
  drop_graph(b);
  return e == cudaSuccess ? MM_OK : bcuda(b, e, "upload work queue");
}

void apply_tune(mm_batch* b, const Tune& t) {
  b->tune = t;
  for (auto& p : b->hp) {
    p.R = best_R(p.g.nv1, p.g.nv2, t.threads);
    p.rows = (t.threads == 32 && p.R == 1 && p.g.nv1 <= 32) ? 1 : 0;
  }
  build_items(b);
}

// Row sums of problem q's g from G itself (after its g was set other than by a sweep, or
// before a tuning that may switch the problem to the row-sum x sweep).
void refresh_rows(mm_batch* b, int q) {
  const BatchProb& d = b->hp[q];
  if (d.g.nv1 <= 32) launch_row_sums(b->G + d.g_off, b->Rm + d.r_off, d.g, b->stream);
}

size_t ctr_words(const mm_batch* b, int nsteps) {
  return 64 + (size_t)nsteps * b->nprob * NPH;
}

mm_status ensure_counters(mm_batch* b, int nsteps) {
  if (nsteps <= b->ctr_steps) return MM_OK;
  drop_graph(b);
  cudaError_t e = cudaStreamSynchronize(b->stream);
  if (e == cudaSuccess) {
    cudaFree(b->d_ctr);
    b->d_ctr = nullptr;
    e = cudaMalloc((void**)&b->d_ctr, sizeof(unsigned) * ctr_words(b, nsteps));
  }
  if (e != cudaSuccess) {
    b->ctr_steps = 0;
    return bcuda(b, e, "work-queue counters");
  }
  b->ctr_steps = nsteps;
  return MM_OK;
}

MegaArgs mega_args(mm_batch* b, double* G, int nsteps) {
  MegaArgs a;
  a.G = G;
  a.Gs = b->Gs;
  a.Q = b->Q;
  a.H = b->H;
  a.prim = b->prim;
  a.mac = b->mac;
  a.Rm = b->Rm;
  a.Ee = b->Ee;
  a.walls = b->walls;
  a.pr = b->d_prob;
  a.items = b->d_items;
  a.need = b->d_need;
  a.head = b->d_ctr;
  a.done = b->d_ctr + 64;
  a.err = b->err;
  a.nitems = (int)b->items.size();
  a.nsteps = nsteps;
  a.nprob = b->nprob;
  a.wait_ns = b->wait_ns;
  a.hold_q = b->hold_q;
  a.hold_ph = b->hold_ph;
  return a;
}

// One launch for nsteps steps: reset the queue and its counters, then the persistent kernel.
void enqueue_steps(mm_batch* b, int nsteps) {
  cudaMemsetAsync(b->d_ctr, 0, sizeof(unsigned) * ctr_words(b, nsteps), b->stream);
  k_batch_steps<<<b->tune.ctas, b->tune.threads, smem_steps(b), b->stream>>>(
      mega_args(b, b->G, nsteps));
}

mm_status upload_desc(mm_batch* b) {
  cudaError_t e = cudaMemcpyAsync(b->d_prob, b->hp.data(), sizeof(BatchProb) * b->nprob,
                                  cudaMemcpyHostToDevice, b->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(b->stream);
  return e == cudaSuccess ? MM_OK : bcuda(b, e, "upload descriptors");
}

// Resident CTAs of the persistent kernel for a CTA size (all SMs x CTAs per SM).
int resident_ctas(const mm_batch* b, int threads) {
  int dev = 0, sms = 152, per_sm = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_batch_steps, threads, smem_steps(b));
  return std::max(1, per_sm) * std::max(1, sms);
}

}  // namespace

extern "C" {

mm_status mm_batch_create(int nprob, const mm_grid* grids, const mm_params* params,
                          void* cuda_stream, mm_batch** out) {
  if (!out || nprob < 1 || !grids || !params) return MM_ERR_INVALID_ARG;
  *out = nullptr;
  for (int q = 0; q < nprob; ++q) {
    if (mm_device_bytes(&grids[q], &params[q]) == 0) return MM_ERR_INVALID_ARG;
    if (params[q].precision != MM_PREC_FP64) return MM_ERR_INVALID_ARG;
    if (grids[q].nv1 > 256) return MM_ERR_INVALID_ARG;
  }
  mm_batch* b = new mm_batch();
  b->nprob = nprob;
  b->grids.assign(grids, grids + nprob);
  b->params.assign(params, params + nprob);
  if (cuda_stream) {
    b->stream = static_cast<cudaStream_t>(cuda_stream);
  } else {
    cudaStreamCreateWithFlags(&b->stream, cudaStreamNonBlocking);
    b->own_stream = true;
  }
  b->hp.resize(nprob);
  b->start.resize(nprob + 1);
  b->wstart.resize(nprob + 1);
  std::vector<int> walls;
  size_t goff = 0, moff = 0, roff = 0, eoff = 0;
  int coff = 0;
  char sig[64];
  std::vector<std::string> shapes;
  for (int q = 0; q < nprob; ++q) {
    const mm_grid& g = grids[q];
    const mm_params& p = params[q];
    BatchProb& d = b->hp[q];
    std::memset(&d, 0, sizeof d);
    d.g.nx = g.nx;
    d.g.ny = g.ny;
    d.g.nv1 = g.nv1;
    d.g.nv2 = g.nv2;
    d.g.dx = (g.x1 - g.x0) / g.nx;
    d.g.dy = (g.y1 - g.y0) / g.ny;
    d.g.idx = 1.0 / d.g.dx;
    d.g.idy = 1.0 / d.g.dy;
    d.g.v1min = g.v1min;
    d.g.v2min = g.v2min;
    d.g.dv1 = (g.v1max - g.v1min) / g.nv1;
    d.g.dv2 = (g.v2max - g.v2min) / g.nv2;
    d.p.nu = p.nu;
    d.p.tau0 = p.tau0;
    d.p.tau_model = p.tau_model;
    for (int s = 0; s < 4; ++s) {
      d.p.bc[s] = p.bc[s];
      d.p.wall_T[s] = p.wall_T[s];
      d.p.wall_U[s] = p.wall_U[s];
    }
    d.p.keep_es = p.wall_keep_es_term ? 1 : 0;
    d.g_off = (long long)goff;
    d.mac_off = (long long)moff;
    d.r_off = (long long)roff;
    d.e_off = (long long)eoff;
    d.c_off = coff;
    d.w_off = (int)walls.size();
    for (int j = 0; j < g.ny; ++j)
      for (int i = 0; i < g.nx; ++i)
        if ((i == 0 && p.bc[0] == MM_BC_DIFFUSE) || (i == g.nx - 1 && p.bc[1] == MM_BC_DIFFUSE) ||
            (j == 0 && p.bc[2] == MM_BC_DIFFUSE) || (j == g.ny - 1 && p.bc[3] == MM_BC_DIFFUSE))
          walls.push_back(j * g.nx + i);
    d.n_wall = (int)walls.size() - d.w_off;
    b->start[q] = coff;
    b->wstart[q] = d.w_off;
    goff += (size_t)g.nx * g.ny * g.nv1 * g.nv2;
    moff += macro_doubles(g.nx, g.ny);
    if (g.nv1 <= 32) roff += (size_t)3 * g.nv1 * g.nx * g.ny;
    eoff += ((size_t)g.nv1 + g.nv2) * g.nx * g.ny;
    coff += g.nx * g.ny;
    b->max_nv1 = std::max(b->max_nv1, g.nv1);
    b->max_nv2 = std::max(b->max_nv2, g.nv2);
    std::snprintf(sig, sizeof sig, "%dx%dx%dx%d", g.nx, g.ny, g.nv1, g.nv2);
    shapes.push_back(sig);
  }
  b->start[nprob] = coff;
  b->wstart[nprob] = (int)walls.size();
  b->nphase = goff;
  b->ncell = coff;
  b->nwall = (int)walls.size();
  std::sort(shapes.begin(), shapes.end());
  for (auto& s : shapes) b->signature += s + ";";

  cudaError_t e = cudaSuccess;
  auto alloc = [&](void** ptr, size_t bytes) {
    if (e == cudaSuccess) e = cudaMalloc(ptr, bytes > 0 ? bytes : 16);
  };
  alloc((void**)&b->G, goff * sizeof(double));
  alloc((void**)&b->Gs, goff * sizeof(double));
  alloc((void**)&b->Q, 6 * (size_t)coff * sizeof(double));
  alloc((void**)&b->H, 4 * (size_t)coff * sizeof(double));
  alloc((void**)&b->prim, NPRIM * (size_t)coff * sizeof(double));
  alloc((void**)&b->mac, moff * sizeof(double));
  alloc((void**)&b->Rm, roff * sizeof(double));
  alloc((void**)&b->Ee, eoff * sizeof(double));
  alloc((void**)&b->walls, walls.size() * sizeof(int));
  alloc((void**)&b->d_prob, nprob * sizeof(BatchProb));
  alloc((void**)&b->err, sizeof(int));
  if (e == cudaSuccess && !walls.empty())
    e = cudaMemcpy(b->walls, walls.data(), walls.size() * sizeof(int), cudaMemcpyHostToDevice);
  if (e == cudaSuccess) e = cudaMemset(b->err, 0, sizeof(int));
  if (e == cudaSuccess) e = cudaMemset(b->G, 0, goff * sizeof(double));
  if (e == cudaSuccess) e = cudaMemset(b->Rm, 0, (roff > 0 ? roff : 2) * sizeof(double));
  if (e != cudaSuccess) {
    mm_batch_destroy(b);
    cudaGetLastError();
    return e == cudaErrorMemoryAllocation ? MM_ERR_OOM : MM_ERR_CUDA;
  }
  if (smem_steps(b) > 48 * 1024)
    cudaFuncSetAttribute(k_batch_steps, cudaFuncAttributeMaxDynamicSharedMemorySize,
                         (int)smem_steps(b));
  // default shape until the autotuner runs: whole warps covering the widest v1 mesh, every
  // resident CTA, one cell per phase-space item and one cell per thread in the per-cell phases
  const int threads = std::max(32, (b->max_nv1 + 31) / 32 * 32);
  Tune t0{threads, resident_ctas(b, threads), 1, threads};
  {
    std::lock_guard<std::mutex> lock(g_tune_mutex);
    auto it = g_tune_cache.find(b->signature);
    if (it != g_tune_cache.end()) t0 = it->second;
  }
  apply_tune(b, t0);
  if (upload_items(b) != MM_OK || ensure_counters(b, 1) != MM_OK) {
    mm_batch_destroy(b);
    return MM_ERR_CUDA;
  }
  b->last_dt.assign(nprob, -1.0);
  b->last_eps.assign(nprob, -1.0);
  *out = b;
  return MM_OK;
}

mm_status mm_batch_set_state(mm_batch* b, int q, const double* Q_host, const double* G_host) {
  if (!b || q < 0 || q >= b->nprob || !Q_host) return bfail(b, MM_ERR_INVALID_ARG, "bad arguments");
  const BatchProb& d = b->hp[q];
  const size_t nc = (size_t)d.g.nx * d.g.ny;
  const size_t np = nc * d.g.nv1 * d.g.nv2;
  cudaError_t e = cudaMemcpyAsync(b->Q + 6 * (size_t)d.c_off, Q_host, 6 * nc * sizeof(double),
                                  cudaMemcpyHostToDevice, b->stream);
  if (e == cudaSuccess) {
    if (G_host)
      e = cudaMemcpyAsync(b->G + d.g_off, G_host, np * sizeof(double), cudaMemcpyHostToDevice,
                          b->stream);
    else
      e = cudaMemsetAsync(b->G + d.g_off, 0, np * sizeof(double), b->stream);
  }
  if (e == cudaSuccess) {
    refresh_rows(b, q);
    e = cudaGetLastError();
  }
  // a new state starts without the device error word of an earlier failed step
  if (e == cudaSuccess) e = cudaMemsetAsync(b->err, 0, sizeof(int), b->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(b->stream);
  return e == cudaSuccess ? MM_OK : bcuda(b, e, "set state");
}

mm_status mm_batch_autotune(mm_batch* b, int* threads_out, int* ctas_out) {
  if (!b) return MM_ERR_INVALID_ARG;
  // trial launches of two whole steps for each candidate tile shape, on the batch's own state,
  // which is saved first and restored afterwards
  const size_t nq = 6 * (size_t)b->ncell, nh = 4 * (size_t)b->ncell;
  size_t nr = 0;
  for (const auto& d : b->hp)
    if (d.g.nv1 <= 32) nr += (size_t)3 * d.g.nv1 * d.g.nx * d.g.ny;
  double* save = nullptr;
  cudaError_t e = cudaMalloc(&save, sizeof(double) * (b->nphase + nq + nh + nr + 1));
  if (e != cudaSuccess) return bcuda(b, e, "autotune buffer");
  double* sG = save;
  double* sQ = sG + b->nphase;
  double* sH = sQ + nq;
  double* sR = sH + nh;
  auto copy_all = [&](bool to_save) {
    auto cp = [&](double* dst, double* src, size_t n) {
      if (n) cudaMemcpyAsync(dst, src, n * sizeof(double), cudaMemcpyDeviceToDevice, b->stream);
    };
    if (to_save) {
      cp(sG, b->G, b->nphase); cp(sQ, b->Q, nq); cp(sH, b->H, nh); cp(sR, b->Rm, nr);
    } else {
      cp(b->G, sG, b->nphase); cp(b->Q, sQ, nq); cp(b->H, sH, nh); cp(b->Rm, sR, nr);
    }
  };
  const Tune cur = b->tune;
  const int T = cur.threads;
  // the row sums of every problem that a candidate may run as one warp per cell
  for (int q = 0; q < b->nprob; ++q) refresh_rows(b, q);
  copy_all(true);
  mm_status st = ensure_counters(b, 2);
  cudaEvent_t e0, e1;
  cudaEventCreate(&e0);
  cudaEventCreate(&e1);
  Tune best = cur;
  float best_ms = 1e30f;
  bool first = true;
  for (int tm : {1, 2, 4, 8})
    for (int tcm : {1, 4}) {
      if (st != MM_OK) break;
      Tune t{T, resident_ctas(b, T), tm, T * tcm};
      apply_tune(b, t);
      st = upload_desc(b);
      if (st == MM_OK) st = upload_items(b);
      if (st != MM_OK) break;
      for (int rep = first ? 0 : 1; rep < 2; ++rep) {  // a warm-up launch before the first
        copy_all(false);
        cudaEventRecord(e0, b->stream);
        enqueue_steps(b, 2);
        cudaEventRecord(e1, b->stream);
        cudaEventSynchronize(e1);
        float ms = 0.f;
        cudaEventElapsedTime(&ms, e0, e1);
        if (rep == 1 && ms < best_ms) {
          best_ms = ms;
          best = t;
        }
      }
      first = false;
    }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  copy_all(false);
  cudaStreamSynchronize(b->stream);
  cudaFree(save);
  cudaMemsetAsync(b->err, 0, sizeof(int), b->stream);
  apply_tune(b, best);
  if (st == MM_OK) st = upload_desc(b);
  if (st == MM_OK) st = upload_items(b);
  {
    std::lock_guard<std::mutex> lock(g_tune_mutex);
    g_tune_cache[b->signature] = best;
  }
  if (threads_out) *threads_out = best.threads;
  if (ctas_out) *ctas_out = best.ctas;
  e = cudaGetLastError();
  if (e != cudaSuccess) return bcuda(b, e, "autotune");
  return st;
}

mm_status mm_batch_tiles(const mm_batch* b, int* micro_cells, int* macro_cells) {
  if (!b) return MM_ERR_INVALID_ARG;
  if (micro_cells) *micro_cells = b->tune.tile_micro;
  if (macro_cells) *macro_cells = b->tune.tile_macro;
  return MM_OK;
}

mm_status mm_batch_diag_hold(mm_batch* b, int q, int phase, double wait_ms) {
  if (!b || q >= b->nprob || phase >= NPH || !(wait_ms > 0.0) || wait_ms > 60000.0)
    return bfail(b, MM_ERR_INVALID_ARG, "bad arguments");
  cudaError_t e = cudaStreamSynchronize(b->stream);
  if (e != cudaSuccess) return bcuda(b, e, "diag hold");
  b->hold_q = q < 0 || phase < 0 ? -1 : q;
  b->hold_ph = q < 0 || phase < 0 ? -1 : phase;
  b->wait_ns = b->hold_q < 0 ? kWaitNs : (long long)(wait_ms * 1e6);
  drop_graph(b);
  return MM_OK;
}

mm_status mm_batch_set_graph(mm_batch* b, int enable) {
  if (!b) return MM_ERR_INVALID_ARG;
  b->use_graph = enable != 0;
  drop_graph(b);
  return MM_OK;
}

mm_status mm_batch_step(mm_batch* b, const double* dt, const double* eps, int nsteps) {
  if (!b || !dt || !eps || nsteps < 0) return bfail(b, MM_ERR_INVALID_ARG, "bad arguments");
  bool changed = false;
  for (int q = 0; q < b->nprob; ++q) {
    if (!(dt[q] > 0.0) || !(eps[q] > 0.0) || !std::isfinite(dt[q]) || !std::isfinite(eps[q]))
      return bfail(b, MM_ERR_INVALID_ARG, "dt and eps must be > 0 for every problem");
    if (dt[q] != b->last_dt[q] || eps[q] != b->last_eps[q]) changed = true;
  }
  if (changed) {
    for (int q = 0; q < b->nprob; ++q) {
      BatchProb& d = b->hp[q];
      d.dt = dt[q];
      d.eps = eps[q];
      d.ieps = 1.0 / eps[q];
      d.dtidx = dt[q] * d.g.idx;
      d.dtidy = dt[q] * d.g.idy;
      d.hscale = eps[q] * d.g.dv1 * d.g.dv2;
      b->last_dt[q] = dt[q];
      b->last_eps[q] = eps[q];
    }
    mm_status st = upload_desc(b);
    if (st != MM_OK) return st;
  }
  if (nsteps == 0) return MM_OK;
  mm_status st = ensure_counters(b, nsteps);
  if (st != MM_OK) return st;
  cudaError_t e = cudaSuccess;
  if (b->use_graph) {
    if (!b->gexec || b->graph_steps != nsteps) {
      drop_graph(b);
      e = cudaStreamBeginCapture(b->stream, cudaStreamCaptureModeThreadLocal);
      if (e != cudaSuccess) return bcuda(b, e, "begin capture");
      enqueue_steps(b, nsteps);
      e = cudaStreamEndCapture(b->stream, &b->graph);
      if (e == cudaSuccess) e = cudaGraphInstantiate(&b->gexec, b->graph, 0);
      if (e != cudaSuccess) {
        drop_graph(b);
        return bcuda(b, e, "graph capture");
      }
      b->graph_steps = nsteps;
    }
    e = cudaGraphLaunch(b->gexec, b->stream);
  } else {
    enqueue_steps(b, nsteps);
    e = cudaGetLastError();
  }
  return e == cudaSuccess ? MM_OK : bcuda(b, e, "batch step");
}

mm_status mm_batch_sync(mm_batch* b) {
  if (!b) return MM_ERR_INVALID_ARG;
  cudaError_t e = cudaStreamSynchronize(b->stream);
  int h = 0;
  if (e == cudaSuccess) e = cudaMemcpy(&h, b->err, sizeof(int), cudaMemcpyDeviceToHost);
  if (e != cudaSuccess) return bcuda(b, e, "batch sync");
  if (h & ERR_WAIT_TIMEOUT)
    return bfail(b, MM_ERR_TIMEOUT, "a bounded wait of the batch work queue ran out");
  if (h) return bfail(b, MM_ERR_NONPHYSICAL, "non-physical state met in a batched problem");
  return MM_OK;
}

mm_status mm_batch_get_moments(mm_batch* b, int q, double* Q_host, double* H_host) {
  if (!b || q < 0 || q >= b->nprob || !Q_host) return bfail(b, MM_ERR_INVALID_ARG, "bad arguments");
  const BatchProb& d = b->hp[q];
  const size_t nc = (size_t)d.g.nx * d.g.ny;
  cudaError_t e = cudaMemcpyAsync(Q_host, b->Q + 6 * (size_t)d.c_off, 6 * nc * sizeof(double),
                                  cudaMemcpyDeviceToHost, b->stream);
  if (e == cudaSuccess && H_host)
    e = cudaMemcpyAsync(H_host, b->H + 4 * (size_t)d.c_off, 4 * nc * sizeof(double),
                        cudaMemcpyDeviceToHost, b->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(b->stream);
  if (e != cudaSuccess) return bcuda(b, e, "get moments");
  return mm_batch_sync(b);
}

mm_status mm_batch_get_g(mm_batch* b, int q, double* G_host) {
  if (!b || q < 0 || q >= b->nprob || !G_host) return bfail(b, MM_ERR_INVALID_ARG, "bad arguments");
  const BatchProb& d = b->hp[q];
  const size_t np = (size_t)d.g.nx * d.g.ny * d.g.nv1 * d.g.nv2;
  cudaError_t e = cudaMemcpyAsync(G_host, b->G + d.g_off, np * sizeof(double),
                                  cudaMemcpyDeviceToHost, b->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(b->stream);
  return e == cudaSuccess ? MM_OK : bcuda(b, e, "get g");
}

const char* mm_batch_last_error(const mm_batch* b) {
  return b ? b->last_error.c_str() : "null batch";
}

void mm_batch_destroy(mm_batch* b) {
  if (!b) return;
  cudaStreamSynchronize(b->stream);
  drop_graph(b);
  cudaFree(b->G);
  cudaFree(b->Gs);
  cudaFree(b->Q);
  cudaFree(b->H);
  cudaFree(b->prim);
  cudaFree(b->mac);
  cudaFree(b->Rm);
  cudaFree(b->Ee);
  cudaFree(b->walls);
  cudaFree(b->d_items);
  cudaFree(b->d_need);
  cudaFree(b->d_ctr);
  cudaFree(b->d_prob);
  cudaFree(b->err);
  if (b->own_stream) cudaStreamDestroy(b->stream);
  delete b;
}

}  // extern "C"
