// Batched stepping of many independent micro-macro KFVS problems of uneven size and Knudsen
// number (Section 5 of Rossmanith & Sar, arXiv 2509.21832, applied to each problem).
//
// All problems live in one set of concatenated device arrays.  Each phase of the step (prims,
// micro x sweep, micro y sweep + relaxation + heat flux, diffuse-wall cells, the three macro
// kernels) is ONE launch of a persistent kernel whose CTAs stride over the cells of all
// problems; a CTA finds the problem of its current cell by binary search in the prefix sums of
// the problems' cell counts and runs the same device body as the single-problem kernels, with
// that problem's grid, parameters, dt and eps read from a descriptor array in device memory.
// One batch step is captured in a CUDA graph and replayed.  The CTA size and the grid size of
// the phase-space kernels are chosen by a small autotuner (timed trial launches on the batch's
// own data), cached per process by the multiset of problem shapes.  Problems that the tuned
// shape runs as one warp per cell with one row per pass keep the row sums of g (sum over v2 of
// v2^j g, j = 0..2, per v1 column) as the single-problem contexts do: the y sweep leaves them
// for the next x sweep, which takes the moments of its upwind differences from them.  No kernel
// waits on another CTA, so there are no spin-waits.
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

__device__ __forceinline__ int find_prob(const int* __restrict__ start, int nprob, int item) {
  int lo = 0, hi = nprob - 1;
  while (lo < hi) {
    const int mid = (lo + hi + 1) >> 1;
    if (__ldg(start + mid) <= item) lo = mid;
    else hi = mid - 1;
  }
  return lo;
}

// Per-cell fields in the two passes of the single-problem step (every cell's (u1, u2, T) first,
// then the rest reading its neighbours' from there), so that every problem of a batch is stepped
// bit for bit as by its own context.
__global__ void k_batch_prims_uT(const double* __restrict__ Q, double* __restrict__ prim,
                                 const BatchProb* __restrict__ pr, const int* __restrict__ start,
                                 int nprob, int total) {
  for (int item = blockIdx.x * blockDim.x + threadIdx.x; item < total;
       item += gridDim.x * blockDim.x) {
    const BatchProb& b = pr[find_prob(start, nprob, item)];
    macro_body::uT_body(Q + 6 * (size_t)b.c_off, prim + NPRIM * (size_t)b.c_off,
                        b.g.nx * b.g.ny, item - b.c_off);
  }
}

__global__ void k_batch_prims(const double* __restrict__ Q, double* __restrict__ prim,
                              const BatchProb* __restrict__ pr, const int* __restrict__ start,
                              int nprob, int total, int* __restrict__ err) {
  for (int item = blockIdx.x * blockDim.x + threadIdx.x; item < total;
       item += gridDim.x * blockDim.x) {
    const BatchProb& b = pr[find_prob(start, nprob, item)];
    macro_body::prims_body<true>(Q + 6 * (size_t)b.c_off, prim + NPRIM * (size_t)b.c_off, nullptr,
                                 b.g, b.p, b.dt, b.eps, b.ieps, err, item - b.c_off);
  }
}

__global__ void k_batch_micro_x(const double* __restrict__ G, double* __restrict__ Gs,
                                const double* __restrict__ prim, const double* __restrict__ Rm,
                                double* __restrict__ Ee, const BatchProb* __restrict__ pr,
                                const int* __restrict__ start, int nprob, int total) {
  extern __shared__ double sm[];
  for (int item = blockIdx.x; item < total; item += gridDim.x) {
    const BatchProb& b = pr[find_prob(start, nprob, item)];
    const double* pp = prim + NPRIM * (size_t)b.c_off;
    if (b.rows)
      micro_body::micro_x_rows_body<double>(G + b.g_off, Gs + b.g_off, pp, Rm + b.r_off,
                                            Ee + b.e_off, b.g, b.p, b.dtidx, item - b.c_off, sm);
    else
      micro_body::micro_x_body<double>(G + b.g_off, Gs + b.g_off, pp, b.g, b.p, b.dtidx, b.R,
                                       item - b.c_off, sm, Ee + b.e_off);
    __syncthreads();
  }
}

__global__ void k_batch_micro_y(const double* __restrict__ Gs, double* __restrict__ G,
                                double* __restrict__ H, const double* __restrict__ prim,
                                double* __restrict__ Rm, const double* __restrict__ Ee,
                                const BatchProb* __restrict__ pr, const int* __restrict__ start,
                                int nprob, int total, int* __restrict__ err) {
  extern __shared__ double sm[];
  for (int item = blockIdx.x; item < total; item += gridDim.x) {
    const BatchProb& b = pr[find_prob(start, nprob, item)];
    micro_body::micro_y_body<double>(Gs + b.g_off, G + b.g_off, H + 4 * (size_t)b.c_off,
                                     prim + NPRIM * (size_t)b.c_off, b.g, b.p, b.dtidy, b.hscale,
                                     b.R, err, item - b.c_off, sm, nullptr, rows_of(Rm, b),
                                     Ee + b.e_off);
    __syncthreads();
  }
}

__global__ void k_batch_micro_y_wall(const double* __restrict__ Gs, double* __restrict__ G,
                                     double* __restrict__ H, const double* __restrict__ prim,
                                     double* __restrict__ Rm, const int* __restrict__ walls,
                                     const BatchProb* __restrict__ pr,
                                     const int* __restrict__ wstart, int nprob, int total,
                                     int* __restrict__ err) {
  extern __shared__ double sm[];
  for (int item = blockIdx.x; item < total; item += gridDim.x) {
    const BatchProb& b = pr[find_prob(wstart, nprob, item)];
    micro_body::micro_y_wall_body<double>(Gs + b.g_off, G + b.g_off, H + 4 * (size_t)b.c_off,
                                          prim + NPRIM * (size_t)b.c_off, b.g, b.p, b.dt, b.eps,
                                          b.R, err, walls[item], sm, rows_of(Rm, b));
    __syncthreads();
  }
}

__global__ void k_batch_macro(int phase, double* __restrict__ Q, const double* __restrict__ H,
                              double* __restrict__ mac, const BatchProb* __restrict__ pr,
                              const int* __restrict__ start, int nprob, int total,
                              int* __restrict__ err) {
  for (int item = blockIdx.x * blockDim.x + threadIdx.x; item < total;
       item += gridDim.x * blockDim.x) {
    const BatchProb& b = pr[find_prob(start, nprob, item)];
    const MacroBufs mb = carve_macro(mac + b.mac_off, b.g.nx, b.g.ny);
    const int c = item - b.c_off;
    double* Qp = Q + 6 * (size_t)b.c_off;
    const double* Hp = H + 4 * (size_t)b.c_off;
    if (phase == 0) macro_body::macro_x1_body(Qp, mb, b.g, b.p, b.dt, b.eps, err, c);
    else if (phase == 1) macro_body::macro_x2_body(Hp, mb, b.g, b.p, b.dt, err, c);
    else macro_body::macro_y_body(Hp, mb, Qp, b.g, b.p, b.dt, b.eps, err, c);
  }
}

struct Tune {
  int threads;
  int ctas;
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
  int* d_start = nullptr;
  int* d_wstart = nullptr;
  BatchProb* d_prob = nullptr;
  int* err = nullptr;
  Tune tune{0, 0};
  bool use_graph = true;
  cudaGraph_t graph = nullptr;
  cudaGraphExec_t gexec = nullptr;
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

size_t smem_x(const mm_batch* b) {
  return sizeof(double) * (micro_body::kRed + 4 * (size_t)b->max_nv2);
}
size_t smem_y(const mm_batch* b) {
  return sizeof(double) * (micro_body::kRed + micro_body::kYTables * (size_t)b->max_nv2);
}
size_t smem_wall(const mm_batch* b) {
  return sizeof(double) * micro_body::wall_smem_doubles(b->max_nv1, b->max_nv2);
}

void apply_tune(mm_batch* b, const Tune& t) {
  b->tune = t;
  for (auto& p : b->hp) {
    p.R = best_R(p.g.nv1, p.g.nv2, t.threads);
    p.rows = (t.threads == 32 && p.R == 1 && p.g.nv1 <= 32) ? 1 : 0;
  }
}

// Row sums of problem q's g from G itself (after its g was set other than by a sweep, or
// before a tuning that may switch the problem to the row-sum x sweep).
void refresh_rows(mm_batch* b, int q) {
  const BatchProb& d = b->hp[q];
  if (d.g.nv1 <= 32) launch_row_sums(b->G + d.g_off, b->Rm + d.r_off, d.g, b->stream);
}

void enqueue_batch_step(mm_batch* b) {
  cudaStream_t s = b->stream;
  const int T = b->tune.threads;
  const int C = b->tune.ctas;
  const int cells = b->ncell;
  const int tb = 256;
  const int cgrid = std::min((cells + tb - 1) / tb, 152 * 16);
  k_batch_prims_uT<<<cgrid, tb, 0, s>>>(b->Q, b->prim, b->d_prob, b->d_start, b->nprob, cells);
  k_batch_prims<<<cgrid, tb, 0, s>>>(b->Q, b->prim, b->d_prob, b->d_start, b->nprob, cells,
                                      b->err);
  k_batch_micro_x<<<C, T, smem_x(b), s>>>(b->G, b->Gs, b->prim, b->Rm, b->Ee, b->d_prob,
                                          b->d_start, b->nprob, cells);
  k_batch_micro_y<<<C, T, smem_y(b), s>>>(b->Gs, b->G, b->H, b->prim, b->Rm, b->Ee, b->d_prob,
                                          b->d_start, b->nprob, cells, b->err);
  if (b->nwall > 0)
    k_batch_micro_y_wall<<<std::min(b->nwall, C), T, smem_wall(b), s>>>(
        b->Gs, b->G, b->H, b->prim, b->Rm, b->walls, b->d_prob, b->d_wstart, b->nprob, b->nwall,
        b->err);
  for (int ph = 0; ph < 3; ++ph)
    k_batch_macro<<<cgrid, tb, 0, s>>>(ph, b->Q, b->H, b->mac, b->d_prob, b->d_start, b->nprob,
                                        cells, b->err);
}

void drop_graph(mm_batch* b) {
  if (b->gexec) cudaGraphExecDestroy(b->gexec);
  if (b->graph) cudaGraphDestroy(b->graph);
  b->gexec = nullptr;
  b->graph = nullptr;
}

mm_status upload_desc(mm_batch* b) {
  cudaError_t e = cudaMemcpyAsync(b->d_prob, b->hp.data(), sizeof(BatchProb) * b->nprob,
                                  cudaMemcpyHostToDevice, b->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(b->stream);
  return e == cudaSuccess ? MM_OK : bcuda(b, e, "upload descriptors");
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
  alloc((void**)&b->d_start, (nprob + 1) * sizeof(int));
  alloc((void**)&b->d_wstart, (nprob + 1) * sizeof(int));
  alloc((void**)&b->d_prob, nprob * sizeof(BatchProb));
  alloc((void**)&b->err, sizeof(int));
  if (e == cudaSuccess && !walls.empty())
    e = cudaMemcpy(b->walls, walls.data(), walls.size() * sizeof(int), cudaMemcpyHostToDevice);
  if (e == cudaSuccess)
    e = cudaMemcpy(b->d_start, b->start.data(), (nprob + 1) * sizeof(int), cudaMemcpyHostToDevice);
  if (e == cudaSuccess)
    e = cudaMemcpy(b->d_wstart, b->wstart.data(), (nprob + 1) * sizeof(int), cudaMemcpyHostToDevice);
  if (e == cudaSuccess) e = cudaMemset(b->err, 0, sizeof(int));
  if (e == cudaSuccess) e = cudaMemset(b->G, 0, goff * sizeof(double));
  if (e == cudaSuccess) e = cudaMemset(b->Rm, 0, (roff > 0 ? roff : 2) * sizeof(double));
  if (e != cudaSuccess) {
    mm_batch_destroy(b);
    cudaGetLastError();
    return e == cudaErrorMemoryAllocation ? MM_ERR_OOM : MM_ERR_CUDA;
  }
  const size_t sm = smem_y(b);
  if (sm > 48 * 1024) {
    cudaFuncSetAttribute(k_batch_micro_y, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
    cudaFuncSetAttribute(k_batch_micro_x, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
  }
  if (smem_wall(b) > 48 * 1024)
    cudaFuncSetAttribute(k_batch_micro_y_wall, cudaFuncAttributeMaxDynamicSharedMemorySize,
                         (int)smem_wall(b));
  // default launch shape until the autotuner runs: whole warps covering the widest v1 mesh
  Tune t0{std::max(32, (b->max_nv1 + 31) / 32 * 32), 152 * 8};
  {
    std::lock_guard<std::mutex> lock(g_tune_mutex);
    auto it = g_tune_cache.find(b->signature);
    if (it != g_tune_cache.end()) t0 = it->second;
  }
  apply_tune(b, t0);
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
  if (e == cudaSuccess) e = cudaStreamSynchronize(b->stream);
  return e == cudaSuccess ? MM_OK : bcuda(b, e, "set state");
}

mm_status mm_batch_autotune(mm_batch* b, int* threads_out, int* ctas_out) {
  if (!b) return MM_ERR_INVALID_ARG;
  // trial launches of the two phase-space kernels on the batch's own data; the y sweep writes
  // into a temporary copy so that the state is untouched
  double* tmp = nullptr;
  cudaError_t e = cudaMalloc(&tmp, b->nphase * sizeof(double));
  if (e != cudaSuccess) return bcuda(b, e, "autotune buffer");
  e = cudaMemcpyAsync(tmp, b->G, b->nphase * sizeof(double), cudaMemcpyDeviceToDevice, b->stream);
  int dev = 0, sms = 152;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  std::vector<int> tcands;
  for (int t : {32, 64, 96, 128, 192, 256})
    if (t >= b->max_nv1) tcands.push_back(t);
  if (tcands.empty()) tcands.push_back((b->max_nv1 + 31) / 32 * 32);
  const int mults[] = {2, 4, 8, 16, 32};
  cudaEvent_t e0, e1;
  cudaEventCreate(&e0);
  cudaEventCreate(&e1);
  Tune best = b->tune;
  float best_ms = 1e30f;
  // the row sums of every problem that a candidate shape may run as one warp per cell (they
  // were not kept for it under the previous shape); the trial y sweeps store none
  for (int q = 0; q < b->nprob; ++q) refresh_rows(b, q);
  // prims once so the coefficient fields are defined (uses the current dt, eps descriptors)
  k_batch_prims_uT<<<std::min((b->ncell + 255) / 256, sms * 16), 256, 0, b->stream>>>(
      b->Q, b->prim, b->d_prob, b->d_start, b->nprob, b->ncell);
  k_batch_prims<<<std::min((b->ncell + 255) / 256, sms * 16), 256, 0, b->stream>>>(
      b->Q, b->prim, b->d_prob, b->d_start, b->nprob, b->ncell, b->err);
  for (int T : tcands)
    for (int m : mults) {
      Tune t{T, m * sms};
      apply_tune(b, t);
      upload_desc(b);
      float total = 0.f;
      for (int rep = 0; rep < 2; ++rep) {
        cudaEventRecord(e0, b->stream);
        k_batch_micro_x<<<t.ctas, t.threads, smem_x(b), b->stream>>>(
            b->G, b->Gs, b->prim, b->Rm, b->Ee, b->d_prob, b->d_start, b->nprob, b->ncell);
        k_batch_micro_y<<<t.ctas, t.threads, smem_y(b), b->stream>>>(
            b->Gs, tmp, b->H, b->prim, nullptr, b->Ee, b->d_prob, b->d_start, b->nprob,
            b->ncell, b->err);
        cudaEventRecord(e1, b->stream);
        cudaEventSynchronize(e1);
        float ms = 0.f;
        cudaEventElapsedTime(&ms, e0, e1);
        if (rep == 1) total = ms;
      }
      if (total < best_ms) {
        best_ms = total;
        best = t;
      }
    }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  cudaFree(tmp);
  cudaMemsetAsync(b->err, 0, sizeof(int), b->stream);
  apply_tune(b, best);
  mm_status st = upload_desc(b);
  drop_graph(b);
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
  cudaError_t e = cudaSuccess;
  if (b->use_graph) {
    if (!b->gexec) {
      e = cudaStreamBeginCapture(b->stream, cudaStreamCaptureModeThreadLocal);
      if (e != cudaSuccess) return bcuda(b, e, "begin capture");
      enqueue_batch_step(b);
      e = cudaStreamEndCapture(b->stream, &b->graph);
      if (e == cudaSuccess) e = cudaGraphInstantiate(&b->gexec, b->graph, 0);
      if (e != cudaSuccess) {
        drop_graph(b);
        return bcuda(b, e, "graph capture");
      }
    }
    for (int n = 0; n < nsteps && e == cudaSuccess; ++n) e = cudaGraphLaunch(b->gexec, b->stream);
  } else {
    for (int n = 0; n < nsteps; ++n) enqueue_batch_step(b);
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
  cudaFree(b->d_start);
  cudaFree(b->d_wstart);
  cudaFree(b->d_prob);
  cudaFree(b->err);
  if (b->own_stream) cudaStreamDestroy(b->stream);
  delete b;
}

}  // extern "C"
