// mm_step_static_scratch: the time step for callers that cannot allocate device memory.
//
// Some callers are not allowed to call cudaMalloc at all: code that runs inside a host
// framework owning every device allocation (a fixed memory budget handed out at start-up),
// plug-ins loaded into such a framework, and real-time loops where allocation after
// initialisation is forbidden.  They can still hand us their own state buffers.  This entry
// point therefore takes Q, G and H in caller-owned device memory and keeps every piece of
// scratch the step needs (the split-step buffer G*, the intermediate macro state Q**, the
// per-cell primitive fields, the diffuse-wall cell list and the error word) in ONE file-scope
// static device array of fixed size.  Every GPU that loads this library holds that array until
// the process exits.
#include <cstdint>
#include <cstdio>
#include <cstring>

#include "mm_internal.cuh"

using namespace mmk;

namespace {

constexpr size_t kAlign = 256;
constexpr size_t round_up(size_t n) { return (n + kAlign - 1) / kAlign * kAlign; }

// Offsets of the regions carved from the static array (bytes, 256-byte aligned).
constexpr size_t kOffGs = 0;
constexpr size_t kOffMacro = kOffGs + round_up(sizeof(double) * MM_STATIC_MAX_PHASE);
// macro buffers: 36 doubles per cell plus 12 per boundary row/column (nx + ny <= cells + 1)
constexpr size_t kOffPrim =
    kOffMacro + round_up(sizeof(double) * (36 * (size_t)MM_STATIC_MAX_CELLS +
                                           12 * ((size_t)MM_STATIC_MAX_CELLS + 1)));
constexpr size_t kOffWall = kOffPrim + round_up(sizeof(double) * NPRIM * MM_STATIC_MAX_CELLS);
constexpr size_t kOffCount = kOffWall + round_up(sizeof(int) * MM_STATIC_MAX_CELLS);
constexpr size_t kOffErr = kOffCount + kAlign;
constexpr size_t kStaticBytes = kOffErr + kAlign;
static_assert(kStaticBytes == MM_STATIC_SCRATCH_BYTES, "header size constant out of date");

// The scratch itself.  In host code this name is only a host-side stand-in for the device
// symbol: host code must use the address from cudaGetSymbolAddress, never the name.
static __device__ __align__(256) unsigned char mm_static_scratch[kStaticBytes];

// Device address of the static array in the current context.  Looked up on every call: the
// lookup allocates nothing, and an address kept from an earlier call could belong to a context
// that has since been destroyed (cudaDeviceReset) or is not the caller's current one.
cudaError_t scratch_address(unsigned char** out) {
  void* p = nullptr;
  cudaError_t e = cudaGetSymbolAddress(&p, mm_static_scratch);
  if (e != cudaSuccess) return e;
  *out = static_cast<unsigned char*>(p);
  return cudaSuccess;
}

__global__ void k_wall_list(int* __restrict__ list, int* __restrict__ count, KGrid g, KParams p) {
  const int c = blockIdx.x * blockDim.x + threadIdx.x;
  if (c >= g.nx * g.ny) return;
  const int i = c % g.nx, j = c / g.nx;
  const bool wall = (i == 0 && p.bc[0] == MM_BC_DIFFUSE) ||
                    (i == g.nx - 1 && p.bc[1] == MM_BC_DIFFUSE) ||
                    (j == 0 && p.bc[2] == MM_BC_DIFFUSE) ||
                    (j == g.ny - 1 && p.bc[3] == MM_BC_DIFFUSE);
  if (wall) list[atomicAdd(count, 1)] = c;
}

mm_status say(char* buf, size_t len, mm_status s, const char* msg) {
  if (buf && len > 0) {
    std::strncpy(buf, msg, len - 1);
    buf[len - 1] = '\0';
  }
  return s;
}

}  // namespace

extern "C" mm_status mm_step_static_scratch(const mm_grid* grid, const mm_params* params,
                                            double* Q_dev, double* G_dev, double* H_dev,
                                            double dt, double eps, int nsteps, void* cuda_stream,
                                            char* errbuf, size_t errlen) {
  if (errbuf && errlen > 0) errbuf[0] = '\0';
  if (mm_device_bytes(grid, params) == 0)
    return say(errbuf, errlen, MM_ERR_INVALID_ARG, "invalid grid or parameters");
  if (params->precision != MM_PREC_FP64)
    return say(errbuf, errlen, MM_ERR_INVALID_ARG, "only MM_PREC_FP64 is supported here");
  const size_t ncell = (size_t)grid->nx * grid->ny;
  const size_t nphase = ncell * grid->nv1 * grid->nv2;
  if (ncell > MM_STATIC_MAX_CELLS || nphase > MM_STATIC_MAX_PHASE) {
    char m[200];
    std::snprintf(m, sizeof m,
                  "problem too large for the static scratch: %zu cells (max %d), %zu phase "
                  "cells (max %d)", ncell, (int)MM_STATIC_MAX_CELLS, nphase,
                  (int)MM_STATIC_MAX_PHASE);
    return say(errbuf, errlen, MM_ERR_INVALID_ARG, m);
  }
  if (!Q_dev || !G_dev || !H_dev)
    return say(errbuf, errlen, MM_ERR_INVALID_ARG, "Q_dev, G_dev and H_dev are required");
  // the same alignment that mm_create_borrowed asks of caller buffers
  if ((uintptr_t)Q_dev % 16 != 0 || (uintptr_t)H_dev % 16 != 0 || (uintptr_t)G_dev % 256 != 0)
    return say(errbuf, errlen, MM_ERR_INVALID_ARG,
               "Q_dev and H_dev must be 16-byte aligned and G_dev 256-byte aligned");
  if (!(dt > 0.0) || !(eps > 0.0) || nsteps < 0)
    return say(errbuf, errlen, MM_ERR_INVALID_ARG, "need dt > 0, eps > 0, nsteps >= 0");

  unsigned char* base = nullptr;
  cudaError_t e = scratch_address(&base);
  if (e != cudaSuccess) return say(errbuf, errlen, MM_ERR_CUDA, cudaGetErrorString(e));

  KGrid kg;
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
  KParams kp;
  kp.nu = params->nu;
  kp.tau0 = params->tau0;
  kp.tau_model = params->tau_model;
  int n_wall = 0;
  for (int s = 0; s < 4; ++s) {
    kp.bc[s] = params->bc[s];
    kp.wall_T[s] = params->wall_T[s];
    kp.wall_U[s] = params->wall_U[s];
  }
  kp.keep_es = params->wall_keep_es_term ? 1 : 0;
  for (int j = 0; j < grid->ny; ++j)
    for (int i = 0; i < grid->nx; ++i)
      if ((i == 0 && kp.bc[0] == MM_BC_DIFFUSE) || (i == grid->nx - 1 && kp.bc[1] == MM_BC_DIFFUSE) ||
          (j == 0 && kp.bc[2] == MM_BC_DIFFUSE) || (j == grid->ny - 1 && kp.bc[3] == MM_BC_DIFFUSE))
        ++n_wall;
  const MicroShape ms = micro_shape(grid->nv1, grid->nv2);

  double* Gs = reinterpret_cast<double*>(base + kOffGs);
  const MacroBufs mb = carve_macro(reinterpret_cast<double*>(base + kOffMacro), grid->nx, grid->ny);
  double* prim = reinterpret_cast<double*>(base + kOffPrim);
  int* wall = reinterpret_cast<int*>(base + kOffWall);
  int* count = reinterpret_cast<int*>(base + kOffCount);
  int* err = reinterpret_cast<int*>(base + kOffErr);
  cudaStream_t s = static_cast<cudaStream_t>(cuda_stream);

  // the array keeps the previous call's contents: clear what must start at zero
  e = cudaMemsetAsync(count, 0, sizeof(int), s);
  if (e == cudaSuccess) e = cudaMemsetAsync(err, 0, sizeof(int), s);
  if (e != cudaSuccess) return say(errbuf, errlen, MM_ERR_CUDA, cudaGetErrorString(e));
  if (n_wall > 0)
    k_wall_list<<<(int)((ncell + 127) / 128), 128, 0, s>>>(wall, count, kg, kp);
  for (int n = 0; n < nsteps; ++n) {
    launch_prims_uT(Q_dev, prim, kg, s);
    launch_prims(Q_dev, prim, nullptr, kg, kp, dt, eps, err, s);
    launch_micro_x<double>(G_dev, Gs, prim, kg, kp, dt, ms, s);
    launch_micro_y<double>(Gs, G_dev, H_dev, prim, kg, kp, dt, eps, ms, err, s);
    launch_micro_y_wall<double>(Gs, G_dev, H_dev, prim, wall, n_wall, kg, kp, dt, eps, ms, err, s);
    launch_macro_x1(Q_dev, mb, kg, kp, dt, eps, err, s);
    launch_macro_x2(H_dev, mb, kg, kp, dt, err, s);
    launch_macro_y(H_dev, mb, Q_dev, kg, kp, dt, eps, err, s);
  }
  e = cudaGetLastError();
  if (e != cudaSuccess) return say(errbuf, errlen, MM_ERR_CUDA, cudaGetErrorString(e));
  int h = 0;
  e = cudaMemcpyAsync(&h, err, sizeof(int), cudaMemcpyDeviceToHost, s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  if (e != cudaSuccess) return say(errbuf, errlen, MM_ERR_CUDA, cudaGetErrorString(e));
  if (h) return say(errbuf, errlen, MM_ERR_NONPHYSICAL, "non-physical state met on the device");
  return MM_OK;
}
