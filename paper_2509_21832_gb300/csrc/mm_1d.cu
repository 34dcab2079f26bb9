// 1D-1V micro-macro scheme for the Boltzmann-BGK equation (Rossmanith & Sar, arXiv 2509.21832,
// Sections 3 and 4): per step
//  - k1d_prims (one thread per cell): rho, u, T of Q^n (E = rho T / 2 + rho u^2 / 2), tau of
//    Eq. (collision_parameter_1d) or a constant, the discrete T_x / T of Eq. (5-19) with the
//    face temperatures of Eqs. (1d_extrap_micro_1/2), (1d_periodic_micro_1/2);
//  - k1d_micro (one CTA per cell): upwind Z (Eq. 5-20), its projection Zhat (Eqs. 5-24, 5-21),
//    Ghat (Eq. 5-19, plus (1/tau)(I - Pi_M)[S] with the manufactured source), the mixed
//    forward/backward Euler update (Eq. 5-25) and the heat flux H^{n+1} (Eq. 5-26);
//  - k1d_macro (one thread per cell): the KFVS update of Eq. (5-27) with the fluxes of Eq.
//    (flux1d_1/2), the boundary rules of Eqs. (1d_extrap_macro_1/2), (1d_periodic_macro), and the
//    manufactured source dt pi^{3/2} cos(2 pi (x - t^n)) (-8, 11, -7) of Section 4.1.
#include <cmath>
#include <string>
#include <utility>
#include <vector>

#include "mm_body_micro.cuh"

namespace {

constexpr double kPi1 = 3.14159265358979323846;

struct K1 {
  int nx, nv;
  double x0, dx, vmin, dv;
  int bc[2];
  int tau_model;
  double tau0;
};

__device__ __forceinline__ double tau_1d(const K1& g, double T) {
  return g.tau_model == MM1D_TAU_HARDSPHERE ? 3.2 * sqrt(T / (2.0 * kPi1)) : g.tau0;
}

__device__ __forceinline__ int nb_1d(const K1& g, int i, int s) {
  const int n = s == 0 ? i - 1 : i + 1;
  if (n >= 0 && n < g.nx) return n;
  if (g.bc[s] == MM_BC_PERIODIC) return (n + g.nx) % g.nx;
  return i;
}

__device__ __forceinline__ void prim_1d(const double* Q, int nx, int i, double& rho, double& u,
                                        double& T) {
  rho = Q[i];
  u = Q[nx + i] / rho;
  T = 2.0 * Q[2 * nx + i] / rho - u * u;
}

// prim [5][nx]: rho, u, T, tau, T_x / T
__global__ void k1d_prims(const double* __restrict__ Q, double* __restrict__ prim, K1 g,
                          int* __restrict__ err) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= g.nx) return;
  const int nx = g.nx;
  double rho, u, T;
  prim_1d(Q, nx, i, rho, u, T);
  if (!(rho > 0.0) || !(T > 0.0) || !isfinite(u) || !isfinite(T)) atomicOr(err, 1);
  double r2, u2, TL, TR;
  prim_1d(Q, nx, nb_1d(g, i, 0), r2, u2, TL);
  prim_1d(Q, nx, nb_1d(g, i, 1), r2, u2, TR);
  const double Tx = (0.5 * (TR + T) - 0.5 * (T + TL)) / (g.dx * T);
  prim[i] = rho;
  prim[nx + i] = u;
  prim[2 * nx + i] = T;
  prim[3 * nx + i] = tau_1d(g, T);
  prim[4 * nx + i] = Tx;
}

// manufactured solution pieces
__device__ __forceinline__ double phi_1d(double v) {
  return exp(-(v - 1.0) * (v - 1.0)) + 2.0 * exp(-(v + 1.0) * (v + 1.0));
}
__device__ __forceinline__ double mex_1d(double v) {
  return 1.8 * exp(-0.04 * (3.0 * v + 1.0) * (3.0 * v + 1.0));
}

// One CTA per cell; thread t handles velocities k = t, t + blockDim.x, ...
__global__ void k1d_micro(const double* __restrict__ G, double* __restrict__ Gn,
                          double* __restrict__ H, const double* __restrict__ prim, K1 g,
                          double dt, double eps, int mms, double tn, int* __restrict__ err) {
  extern __shared__ double red[];  // block_sum4 scratch
  const int nx = g.nx, nv = g.nv;
  const int i = blockIdx.x;
  const int iL = nb_1d(g, i, 0), iR = nb_1d(g, i, 1);
  const bool left_ok = !(i == 0 && g.bc[0] != MM_BC_PERIODIC);
  const bool right_ok = !(i == nx - 1 && g.bc[1] != MM_BC_PERIODIC);
  const double rho = prim[i], u = prim[nx + i], T = prim[2 * nx + i];
  const double tau = prim[3 * nx + i], Tx = prim[4 * nx + i];
  const double sT = sqrt(T), isT = 1.0 / sT, r2 = sqrt(2.0);
  const double Mk = rho / sqrt(2.0 * kPi1 * T);
  const double* Gc = G + (size_t)i * nv;
  const double* Gl = G + (size_t)iL * nv;
  const double* Gr = G + (size_t)iR * nv;
  // manufactured source at (x_i, t^n): S = phi (F_t + v F_x) - (tau_e/eps)(M_e - phi) F with the
  // exact state's Maxwellian M_e and tau_e = tau(T = 25/18): S is a function of (t, x, v) alone
  const double x = g.x0 + (i + 0.5) * g.dx;
  const double F = 2.0 + sin(2.0 * kPi1 * (x - tn));
  const double Fx = 2.0 * kPi1 * cos(2.0 * kPi1 * (x - tn));
  const double te = tau_1d(g, 25.0 / 18.0) / eps;
  // pass 1: moments of Z (and of S) against the basis of Eq. (5-5)
  double a[4] = {0, 0, 0, 0}, b[4] = {0, 0, 0, 0};
  for (int k = threadIdx.x; k < nv; k += blockDim.x) {
    const double v = fma(k + 0.5, g.dv, g.vmin);
    const double gc = Gc[k];
    double z = 0.0;
    if (right_ok && v < 0.0) z += v * (Gr[k] - gc) / g.dx;
    if (left_ok && v > 0.0) z += v * (gc - Gl[k]) / g.dx;
    const double c = (v - u) * isT;
    const double b3 = r2 * (0.5 * c * c - 0.5);
    a[0] += z;
    a[1] = fma(c, z, a[1]);
    a[2] = fma(b3, z, a[2]);
    if (mms) {
      const double ph = phi_1d(v);
      const double S = ph * (-Fx + v * Fx) - te * (mex_1d(v) - ph) * F;
      b[0] += S;
      b[1] = fma(c, S, b[1]);
      b[2] = fma(b3, S, b[2]);
    }
  }
  mmk::micro_body::block_sum4(a, red);
  if (mms) mmk::micro_body::block_sum4(b, red);
  const double sc = g.dv / rho;
  const double A1 = a[0] * sc, A2 = a[1] * sc, A3 = a[2] * sc;
  const double B1 = b[0] * sc, B2 = b[1] * sc, B3 = b[2] * sc;
  const double w1 = eps / (eps + dt * tau), w2 = dt * tau / (eps + dt * tau);
  // pass 2: Zhat, Ghat, G^{n+1} and the heat flux
  double h[4] = {0, 0, 0, 0};
  double* Go = Gn + (size_t)i * nv;
  for (int k = threadIdx.x; k < nv; k += blockDim.x) {
    const double v = fma(k + 0.5, g.dv, g.vmin);
    const double gc = Gc[k];
    double z = 0.0;
    if (right_ok && v < 0.0) z += v * (Gr[k] - gc) / g.dx;
    if (left_ok && v > 0.0) z += v * (gc - Gl[k]) / g.dx;
    const double cu = v - u;
    const double c = cu * isT;
    const double b3 = r2 * (0.5 * c * c - 0.5);
    const double M = Mk * exp(-cu * cu / (2.0 * T));
    const double zh = (A1 + c * A2 + b3 * A3) * M;
    double gh = -(1.0 / tau) * (cu * cu * cu / (2.0 * T) - 1.5 * cu) * Tx * M;
    if (mms) {
      const double ph = phi_1d(v);
      const double S = ph * (-Fx + v * Fx) - te * (mex_1d(v) - ph) * F;
      gh += (S - (B1 + c * B2 + b3 * B3) * M) / tau;
    }
    const double gn = w1 * (gc - dt * (z - zh)) + w2 * gh;
    Go[k] = gn;
    h[0] = fma(v * v * v, gn, h[0]);
  }
  mmk::micro_body::block_sum4(h, red);
  if (threadIdx.x == 0) {
    H[i] = 0.5 * eps * g.dv * h[0];
    if (!isfinite(h[0])) atomicOr(err, 4);
  }
}

__device__ __forceinline__ void kfvs_1d(double rho, double u, double T, double Fp[3],
                                        double Fm[3]) {
  const double a = sqrt(T / (2.0 * kPi1)) * exp(-u * u / (2.0 * T));
  const double e = erf(u / sqrt(2.0 * T));
  const double bp = 0.5 * (1.0 + e), bm = 0.5 * (1.0 - e);
  const double w[3] = {rho, rho * u, 0.5 * rho * (2.0 * T + u * u)};
  const double f[3] = {rho * u, rho * (T + u * u), 0.5 * rho * u * (3.0 * T + u * u)};
  for (int m = 0; m < 3; ++m) {
    Fp[m] = a * w[m] + bp * f[m];
    Fm[m] = -a * w[m] + bm * f[m];
  }
}

__global__ void k1d_macro(const double* __restrict__ Q, double* __restrict__ Qn,
                          const double* __restrict__ H, const double* __restrict__ prim, K1 g,
                          double dt, int mms, double tn, int* __restrict__ err) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= g.nx) return;
  const int nx = g.nx;
  const int iL = nb_1d(g, i, 0), iR = nb_1d(g, i, 1);
  double Fp[3], Fm[3], Gp[3], Gm[3], FL[3], FR[3];
  kfvs_1d(prim[i], prim[nx + i], prim[2 * nx + i], Fp, Fm);
  double HL, HR;
  if (i == 0 && g.bc[0] != MM_BC_PERIODIC) {
    for (int m = 0; m < 3; ++m) FL[m] = Fp[m] + Fm[m];
    HL = H[i];
  } else {
    kfvs_1d(prim[iL], prim[nx + iL], prim[2 * nx + iL], Gp, Gm);
    for (int m = 0; m < 3; ++m) FL[m] = Gp[m] + Fm[m];
    HL = 0.5 * (H[i] + H[iL]);
  }
  if (i == nx - 1 && g.bc[1] != MM_BC_PERIODIC) {
    for (int m = 0; m < 3; ++m) FR[m] = Fp[m] + Fm[m];
    HR = H[i];
  } else {
    kfvs_1d(prim[iR], prim[nx + iR], prim[2 * nx + iR], Gp, Gm);
    for (int m = 0; m < 3; ++m) FR[m] = Fp[m] + Gm[m];
    HR = 0.5 * (H[iR] + H[i]);
  }
  const double lam = dt / g.dx;
  double q[3];
  for (int m = 0; m < 3; ++m) q[m] = Q[m * nx + i] - lam * (FR[m] - FL[m]);
  q[2] -= lam * (HR - HL);
  if (mms) {
    const double c = pow(kPi1, 1.5) * cos(2.0 * kPi1 * (g.x0 + (i + 0.5) * g.dx - tn));
    q[0] += dt * c * -8.0;
    q[1] += dt * c * 11.0;
    q[2] += dt * c * -7.0;
  }
  for (int m = 0; m < 3; ++m) Qn[m * nx + i] = q[m];
  if (!(q[0] > 0.0) || !isfinite(q[1]) || !isfinite(q[2])) atomicOr(err, 2);
}

__global__ void k1d_exact(double* __restrict__ Q, double* __restrict__ G, K1 g, double t,
                          double eps) {
  const int i = blockIdx.x;
  const double F = 2.0 + sin(2.0 * kPi1 * (g.x0 + (i + 0.5) * g.dx - t));
  if (threadIdx.x == 0) {
    const double rho = 3.0 * sqrt(kPi1) * F, u = -1.0 / 3.0, T = 25.0 / 18.0;
    Q[i] = rho;
    Q[g.nx + i] = rho * u;
    Q[2 * g.nx + i] = 0.5 * rho * T + 0.5 * rho * u * u;
  }
  for (int k = threadIdx.x; k < g.nv; k += blockDim.x) {
    const double v = fma(k + 0.5, g.dv, g.vmin);
    G[(size_t)i * g.nv + k] = (phi_1d(v) - mex_1d(v)) * F / eps;
  }
}

int threads_1d(int nv) { return nv >= 256 ? 256 : (nv + 31) / 32 * 32; }

}  // namespace

struct mm1d_ctx {
  K1 g{};
  cudaStream_t stream = nullptr;
  double *Q = nullptr, *Qn = nullptr, *G = nullptr, *Gn = nullptr, *H = nullptr;
  double* prim = nullptr;
  int* err = nullptr;
  bool mms = false;
  double t = 0.0;
  bool have_state = false;
  std::string last_error;
};

namespace {
mm_status f1(mm1d_ctx* c, mm_status s, const std::string& m) {
  if (c) c->last_error = m;
  return s;
}
mm_status c1(mm1d_ctx* c, cudaError_t e, const char* what) {
  return f1(c, MM_ERR_CUDA, std::string(what) + ": " + cudaGetErrorString(e));
}
mm_status sync_check(mm1d_ctx* c) {
  int h = 0;
  cudaError_t e = cudaMemcpyAsync(&h, c->err, sizeof(int), cudaMemcpyDeviceToHost, c->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
  if (e != cudaSuccess) return c1(c, e, "synchronize");
  if (h) return f1(c, MM_ERR_NONPHYSICAL, "non-physical state met on the device");
  return MM_OK;
}
}  // namespace

extern "C" {

mm_status mm1d_create(const mm1d_grid* grid, const mm1d_params* params, void* cuda_stream,
                      mm1d_ctx** out) {
  if (!out) return MM_ERR_INVALID_ARG;
  *out = nullptr;
  if (!grid || !params || grid->nx < 2 || grid->nv < 1 || grid->nv > 65536 ||
      !(grid->x1 > grid->x0) || !(grid->vmax > grid->vmin))
    return MM_ERR_INVALID_ARG;
  for (int s = 0; s < 2; ++s)
    if (params->bc[s] != MM_BC_PERIODIC && params->bc[s] != MM_BC_EXTRAP) return MM_ERR_INVALID_ARG;
  if ((params->bc[0] == MM_BC_PERIODIC) != (params->bc[1] == MM_BC_PERIODIC)) return MM_ERR_INVALID_ARG;
  if (params->tau_model != MM1D_TAU_HARDSPHERE &&
      !(params->tau_model == MM1D_TAU_CONST && params->tau0 > 0.0))
    return MM_ERR_INVALID_ARG;
  mm1d_ctx* c = new mm1d_ctx();
  c->stream = static_cast<cudaStream_t>(cuda_stream);
  K1& g = c->g;
  g.nx = grid->nx;
  g.nv = grid->nv;
  g.x0 = grid->x0;
  g.dx = (grid->x1 - grid->x0) / grid->nx;
  g.vmin = grid->vmin;
  g.dv = (grid->vmax - grid->vmin) / grid->nv;
  g.bc[0] = params->bc[0];
  g.bc[1] = params->bc[1];
  g.tau_model = params->tau_model;
  g.tau0 = params->tau0;
  const size_t np = (size_t)g.nx * g.nv;
  cudaError_t e = cudaMalloc(&c->Q, 3 * g.nx * sizeof(double));
  if (e == cudaSuccess) e = cudaMalloc(&c->Qn, 3 * g.nx * sizeof(double));
  if (e == cudaSuccess) e = cudaMalloc(&c->G, np * sizeof(double));
  if (e == cudaSuccess) e = cudaMalloc(&c->Gn, np * sizeof(double));
  if (e == cudaSuccess) e = cudaMalloc(&c->H, g.nx * sizeof(double));
  if (e == cudaSuccess) e = cudaMalloc(&c->prim, 5 * g.nx * sizeof(double));
  if (e == cudaSuccess) e = cudaMalloc(&c->err, sizeof(int));
  if (e == cudaSuccess) e = cudaMemsetAsync(c->err, 0, sizeof(int), c->stream);
  if (e == cudaSuccess) e = cudaMemsetAsync(c->H, 0, g.nx * sizeof(double), c->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
  if (e != cudaSuccess) {
    mm1d_destroy(c);
    return e == cudaErrorMemoryAllocation ? MM_ERR_OOM : MM_ERR_CUDA;
  }
  *out = c;
  return MM_OK;
}

mm_status mm1d_set_state(mm1d_ctx* c, const double* Q_host, const double* G_host) {
  if (!c) return MM_ERR_INVALID_ARG;
  if (!Q_host) return f1(c, MM_ERR_INVALID_ARG, "Q_host is NULL");
  const size_t np = (size_t)c->g.nx * c->g.nv;
  cudaError_t e = cudaMemcpyAsync(c->Q, Q_host, 3 * c->g.nx * sizeof(double),
                                  cudaMemcpyHostToDevice, c->stream);
  if (e == cudaSuccess)
    e = G_host ? cudaMemcpyAsync(c->G, G_host, np * sizeof(double), cudaMemcpyHostToDevice, c->stream)
               : cudaMemsetAsync(c->G, 0, np * sizeof(double), c->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
  if (e != cudaSuccess) return c1(c, e, "set state");
  c->have_state = true;
  return MM_OK;
}

mm_status mm1d_step(mm1d_ctx* c, double dt, double eps, int nsteps) {
  if (!c) return MM_ERR_INVALID_ARG;
  if (!(dt > 0.0) || !(eps > 0.0) || nsteps < 0) return f1(c, MM_ERR_INVALID_ARG, "bad dt, eps or nsteps");
  if (!c->have_state) return f1(c, MM_ERR_STATE, "no state set");
  const K1& g = c->g;
  const int th = threads_1d(g.nv);
  for (int n = 0; n < nsteps; ++n) {
    k1d_prims<<<(g.nx + 127) / 128, 128, 0, c->stream>>>(c->Q, c->prim, g, c->err);
    k1d_micro<<<g.nx, th, sizeof(double) * mmk::micro_body::kRed, c->stream>>>(
        c->G, c->Gn, c->H, c->prim, g, dt, eps, c->mms ? 1 : 0, c->t, c->err);
    k1d_macro<<<(g.nx + 127) / 128, 128, 0, c->stream>>>(c->Q, c->Qn, c->H, c->prim, g, dt,
                                                         c->mms ? 1 : 0, c->t, c->err);
    std::swap(c->G, c->Gn);
    std::swap(c->Q, c->Qn);
    c->t += dt;
  }
  cudaError_t e = cudaGetLastError();
  return e == cudaSuccess ? MM_OK : c1(c, e, "kernel launch");
}

mm_status mm1d_get_state(mm1d_ctx* c, double* Q_host, double* G_host, double* H_host) {
  if (!c) return MM_ERR_INVALID_ARG;
  const size_t np = (size_t)c->g.nx * c->g.nv;
  cudaError_t e = cudaSuccess;
  if (Q_host) e = cudaMemcpyAsync(Q_host, c->Q, 3 * c->g.nx * sizeof(double), cudaMemcpyDeviceToHost, c->stream);
  if (e == cudaSuccess && G_host)
    e = cudaMemcpyAsync(G_host, c->G, np * sizeof(double), cudaMemcpyDeviceToHost, c->stream);
  if (e == cudaSuccess && H_host)
    e = cudaMemcpyAsync(H_host, c->H, c->g.nx * sizeof(double), cudaMemcpyDeviceToHost, c->stream);
  if (e != cudaSuccess) return c1(c, e, "copy state out");
  return sync_check(c);
}

mm_status mm1d_mms_enable(mm1d_ctx* c, int enable, double t0) {
  if (!c) return MM_ERR_INVALID_ARG;
  if (enable && (c->g.bc[0] != MM_BC_PERIODIC || !std::isfinite(t0)))
    return f1(c, MM_ERR_INVALID_ARG, "the manufactured solution is periodic; t0 must be finite");
  c->mms = enable != 0;
  c->t = t0;
  return MM_OK;
}

mm_status mm1d_mms_set_exact(mm1d_ctx* c, double t, double eps) {
  if (!c) return MM_ERR_INVALID_ARG;
  if (!(eps > 0.0) || !std::isfinite(t)) return f1(c, MM_ERR_INVALID_ARG, "bad t or eps");
  k1d_exact<<<c->g.nx, threads_1d(c->g.nv), 0, c->stream>>>(c->Q, c->G, c->g, t, eps);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return c1(c, e, "exact state");
  c->have_state = true;
  return MM_OK;
}

const char* mm1d_last_error(const mm1d_ctx* c) { return c ? c->last_error.c_str() : "null context"; }

void mm1d_destroy(mm1d_ctx* c) {
  if (!c) return;
  cudaStreamSynchronize(c->stream);
  cudaFree(c->Q);
  cudaFree(c->Qn);
  cudaFree(c->G);
  cudaFree(c->Gn);
  cudaFree(c->H);
  cudaFree(c->prim);
  cudaFree(c->err);
  delete c;
}

}  // extern "C"
