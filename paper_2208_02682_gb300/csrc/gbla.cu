// gbla.cu -- semi-Lagrangian discretisation of Strategy 1 (App. B): the
// grid-based Lagrangian average, advanced after every RK4 step of a handle's
// dynamics on FP64 physical grid fields.
//
// Per grid point X (one thread), with the departure point Y = X - dt u(X,
// t_{n+1}) taken as a displacement from the node:
//   backward Euler   g(X) = g_I(Y) + dt f(X)                 Eq. (sdiscrete_gtilde)
//   trapezoidal      g(X) = g_I(Y) + dt [f_I(Y, t_n) + f(X)]/2
//                                             Eq. (sdiscrete_gtilde_trapez)
//   positions        D(X) = D_I(Y) + (s_n + w dt) dt u(X)
// (D = s (x - Xi^{-1}), the rule applied to f = x: Eq. (sdiscrete_Xi-1) for
// the trapezoid, w = 1/2; w = 0 for backward Euler).  Interpolation:
// bilinear, or tensor-product 4-point Lagrange on the cells i-1 .. i+2.
// Fields and displacements are double-buffered (a point reads its
// neighbours' old values).
#include <cuda_runtime.h>

#include <cmath>
#include <cstring>
#include <new>
#include <string>

#include "../../include/lagmean.h"
#include "launch.cuh"

using namespace lm;

namespace lm {
void set_handleless_error(const std::string& msg);
}

namespace {

constexpr double kTwoPi = 6.283185307179586476925286766559;
constexpr int kMaxSL = 5;  // zeta, h, u, v, q

// physical source of each averaged scalar, in LM_* bit order: the staging
// slots hold u, v, h, zeta; q is formed from zeta and h
enum { SRC_ZETA = 3, SRC_H = 2, SRC_U = 0, SRC_V = 1, SRC_Q = 4 };

struct SLArgs {
  const double* phys;  // u, v, h, zeta at t_{n+1}, N*N each
  const double* g0;    // g at t_n (nf fields)
  double* g1;          // g at t_{n+1}
  const double* f0;    // f at t_n (trapezoid)
  double* f1;          // f at t_{n+1} (trapezoid)
  const double* d0;    // D at t_n (2 components)
  double* d1;
  int src[kMaxSL];
  int N, log2N, nf, cubic, trap, pos, kin;
  double dt, s_n, fcor, adv_x, adv_y;
};

struct Stencil {
  int i[4], j[4];  // columns and rows i0-1 .. i0+2 (periodic)
  double wx[4], wy[4];
  bool cubic;
};

__device__ __forceinline__ void lagrange4(double a, double* w) {
  w[0] = -a * (a - 1.0) * (a - 2.0) / 6.0;
  w[1] = (a + 1.0) * (a - 1.0) * (a - 2.0) / 2.0;
  w[2] = -(a + 1.0) * a * (a - 2.0) / 2.0;
  w[3] = (a + 1.0) * a * (a - 1.0) / 6.0;
}

__device__ __forceinline__ Stencil stencil(int i, int j, double ddx, double ddy, int N, bool cubic) {
  const double inv_dx = (double)N / kTwoPi;
  const double cx = ddx * inv_dx, cy = ddy * inv_dx;
  const double fx = floor(cx), fy = floor(cy);
  const double ax = cx - fx, ay = cy - fy;
  const unsigned msk = (unsigned)N - 1u;
  const unsigned i0 = ((unsigned)i + (unsigned)(long long)fx) & msk;
  const unsigned j0 = ((unsigned)j + (unsigned)(long long)fy) & msk;
  Stencil s;
  s.cubic = cubic;
#pragma unroll
  for (int q = 0; q < 4; ++q) {
    s.i[q] = (int)((i0 + (unsigned)(q - 1)) & msk);
    s.j[q] = (int)((j0 + (unsigned)(q - 1)) & msk);
  }
  if (cubic) {
    lagrange4(ax, s.wx);
    lagrange4(ay, s.wy);
  } else {
    s.wx[0] = s.wx[3] = s.wy[0] = s.wy[3] = 0.0;
    s.wx[1] = 1.0 - ax;
    s.wx[2] = ax;
    s.wy[1] = 1.0 - ay;
    s.wy[2] = ay;
  }
  return s;
}

__device__ __forceinline__ double interp(const double* __restrict__ f, const Stencil& s, int N) {
  if (!s.cubic) {
    const double* r0 = f + (long long)s.j[1] * N;
    const double* r1 = f + (long long)s.j[2] * N;
    return s.wx[1] * s.wy[1] * r0[s.i[1]] + s.wx[2] * s.wy[1] * r0[s.i[2]] + s.wx[1] * s.wy[2] * r1[s.i[1]] +
           s.wx[2] * s.wy[2] * r1[s.i[2]];
  }
  double out = 0.0;
#pragma unroll
  for (int q = 0; q < 4; ++q) {
    const double* row = f + (long long)s.j[q] * N;
    double acc = 0.0;
#pragma unroll
    for (int p = 0; p < 4; ++p) acc += s.wx[p] * row[s.i[p]];
    out += s.wy[q] * acc;
  }
  return out;
}

__device__ __forceinline__ double source(const SLArgs& a, int src, long long idx, long long np) {
  if (src == SRC_Q) return (a.fcor + a.phys[3 * np + idx]) / a.phys[2 * np + idx];
  return a.phys[src * np + idx];
}

__global__ void __launch_bounds__(256) k_sl_step(const __grid_constant__ SLArgs a) {
  const int N = a.N;
  const long long np = (long long)N * N;
  const long long idx = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= np) return;
  const int i = (int)(idx & (N - 1)), j = (int)(idx >> a.log2N);
  const double ux = a.kin ? a.adv_x : a.phys[idx];
  const double uy = a.kin ? a.adv_y : a.phys[np + idx];
  const Stencil s = stencil(i, j, -a.dt * ux, -a.dt * uy, N, a.cubic);
  for (int k = 0; k < a.nf; ++k) {
    const double fx = source(a, a.src[k], idx, np);
    const double gy = interp(a.g0 + k * np, s, N);
    if (a.trap) {
      a.g1[k * np + idx] = gy + a.dt * (interp(a.f0 + k * np, s, N) + fx) / 2.0;
      a.f1[k * np + idx] = fx;
    } else {
      a.g1[k * np + idx] = gy + a.dt * fx;
    }
  }
  if (a.pos) {
    const double c = (a.s_n + (a.trap ? 0.5 : 0.0) * a.dt) * a.dt;
    a.d1[idx] = interp(a.d0, s, N) + c * ux;
    a.d1[np + idx] = interp(a.d0 + np, s, N) + c * uy;
  }
}

// f at tau for the trapezoid's first step
__global__ void k_sl_init(SLArgs a) {
  const long long np = (long long)a.N * a.N;
  const long long idx = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= np) return;
  for (int k = 0; k < a.nf; ++k) a.f1[k * np + idx] = source(a, a.src[k], idx, np);
}

// results: f~^L = g/T into out (nf fields), Xi^{-1} = x - D/T into pos
__global__ void k_sl_out(const double* g, const double* d, double* out, double* pos, int N, int log2N, int nf,
                         int want_pos, double T) {
  const long long np = (long long)N * N;
  const long long idx = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= np) return;
  for (int k = 0; k < nf; ++k) out[k * np + idx] = g[k * np + idx] / T;
  if (want_pos) {
    const int i = (int)(idx & (N - 1)), j = (int)(idx >> log2N);
    pos[idx] = kTwoPi * i / N - d[idx] / T;
    pos[np + idx] = kTwoPi * j / N - d[np + idx] / T;
  }
}

}  // namespace

struct sl_interval {
  sw_handle* h = nullptr;
  sl_params p{};
  HandleInfo hi{};
  int log2N = 0;
  int nf = 0;
  int src[kMaxSL] = {};
  int bit[kMaxSL] = {};
  bool pos = false;
  int64_t done = 0;
  double* arena = nullptr;
  double *g[2] = {}, *f[2] = {}, *d[2] = {};
  int cur = 0;
};

static int sl_fail(sw_handle* h, int rc, const std::string& m) {
  if (h) handle_set_error(h, "sw_sl: " + m);
  else set_handleless_error("sw_sl: " + m);
  return rc;
}

static SLArgs sl_args(sl_interval* s, const double* phys) {
  SLArgs a;
  std::memset(&a, 0, sizeof(a));
  a.phys = phys;
  const int c = s->cur, n = s->cur ^ 1;
  a.g0 = s->g[c];
  a.g1 = s->g[n];
  a.f0 = s->f[c];
  a.f1 = s->f[n];
  a.d0 = s->d[c];
  a.d1 = s->d[n];
  for (int k = 0; k < s->nf; ++k) a.src[k] = s->src[k];
  a.N = s->hi.N;
  a.log2N = s->log2N;
  a.nf = s->nf;
  a.cubic = s->p.interp == SL_CUBIC;
  a.trap = s->p.scheme == SL_TRAPEZOID;
  a.pos = s->pos;
  a.kin = s->hi.model == SW_MODEL_KINEMATIC;
  a.dt = s->hi.dt;
  a.s_n = (double)s->done * s->hi.dt;
  a.fcor = s->hi.f0;
  a.adv_x = s->hi.adv_x;
  a.adv_y = s->hi.adv_y;
  return a;
}

extern "C" int sw_sl_create(sw_handle* h, const sl_params* p, sl_interval** out) {
  if (!out) return sl_fail(h, SW_EINVAL, "out is NULL");
  *out = nullptr;
  if (!h) return sl_fail(nullptr, SW_EINVAL, "handle is NULL");
  if (!p) return sl_fail(h, SW_EINVAL, "params is NULL");
  const int known = LM_ZETA | LM_H | LM_U | LM_V | LM_Q | LM_POS;
  if (p->fields == 0 || (p->fields & ~known)) return sl_fail(h, SW_EINVAL, "fields must be a nonzero LM_* mask");
  if (p->scheme != SL_EULER && p->scheme != SL_TRAPEZOID) return sl_fail(h, SW_EINVAL, "unknown scheme");
  if (p->interp != SL_LINEAR && p->interp != SL_CUBIC) return sl_fail(h, SW_EINVAL, "unknown interpolation");
  if (p->reserved != 0) return sl_fail(h, SW_EINVAL, "reserved must be 0");
  if (p->n_steps < 1) return sl_fail(h, SW_EINVAL, "n_steps must be >= 1");
  sl_interval* s = new (std::nothrow) sl_interval();
  if (!s) return sl_fail(h, SW_ENOMEM, "host allocation failed");
  s->h = h;
  s->p = *p;
  int rc = handle_info(h, &s->hi);
  if (rc) {
    delete s;
    return sl_fail(h, rc, "handle query failed");
  }
  if (s->hi.lm_open) {
    delete s;
    return sl_fail(h, SW_EBUSY, "the handle has an open averaging interval");
  }
  if (s->hi.model == SW_MODEL_EULER2D && (p->fields & (LM_H | LM_Q))) {
    delete s;
    return sl_fail(h, SW_EINVAL, "the two-dimensional Euler model averages zeta, u and v only");
  }
  while ((1 << s->log2N) < s->hi.N) ++s->log2N;
  const int bits[kMaxSL] = {LM_ZETA, LM_H, LM_U, LM_V, LM_Q};
  const int srcs[kMaxSL] = {SRC_ZETA, SRC_H, SRC_U, SRC_V, SRC_Q};
  for (int k = 0; k < kMaxSL; ++k)
    if (p->fields & bits[k]) {
      s->bit[s->nf] = bits[k];
      s->src[s->nf++] = srcs[k];
    }
  s->pos = (p->fields & LM_POS) != 0;
  const size_t np = (size_t)s->hi.N * s->hi.N;
  const size_t nf = (size_t)(s->nf > 0 ? s->nf : 1);
  const size_t per = 2 * nf * np + 2 * nf * np + 2 * 2 * np;  // g, f, d: two buffers each
  cudaError_t e = cudaMalloc(&s->arena, per * sizeof(double));
  if (e != cudaSuccess) {
    cudaGetLastError();
    delete s;
    return sl_fail(h, SW_ENOMEM, std::string("cudaMalloc: ") + cudaGetErrorString(e));
  }
  double* q = s->arena;
  for (int b = 0; b < 2; ++b) {
    s->g[b] = q;
    q += nf * np;
    s->f[b] = q;
    q += nf * np;
    s->d[b] = q;
    q += 2 * np;
  }
  cudaStream_t st = s->hi.stream;
  e = cudaMemsetAsync(s->arena, 0, per * sizeof(double), st);
  if (e == cudaSuccess && p->scheme == SL_TRAPEZOID && s->nf > 0) {
    const double* phys = nullptr;
    rc = handle_phys_uvhz(h, &phys);
    if (rc) {
      cudaFree(s->arena);
      delete s;
      return rc;
    }
    SLArgs a = sl_args(s, phys);
    a.f1 = s->f[s->cur];  // f at tau is read by the first step
    k_sl_init<<<(unsigned)((np + 255) / 256), 256, 0, st>>>(a);
    e = cudaGetLastError();
  }
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  if (e != cudaSuccess) {
    cudaFree(s->arena);
    delete s;
    return sl_fail(h, SW_ECUDA, std::string("set-up: ") + cudaGetErrorString(e));
  }
  *out = s;
  return SW_OK;
}

extern "C" int sw_sl_step(sl_interval* s, int64_t nsteps) {
  if (!s) return SW_EINVAL;
  if (nsteps < 0) return sl_fail(s->h, SW_EINVAL, "nsteps must be >= 0");
  if (nsteps > s->p.n_steps - s->done) return sl_fail(s->h, SW_ERANGE, "more steps than remain in the interval");
  const long long np = (long long)s->hi.N * s->hi.N;
  for (int64_t it = 0; it < nsteps; ++it) {
    int rc = sw_step(s->h, 1);
    if (rc) return rc;
    const double* phys = nullptr;
    rc = handle_phys_uvhz(s->h, &phys);
    if (rc) return rc;
    const SLArgs a = sl_args(s, phys);
    k_sl_step<<<(unsigned)((np + 255) / 256), 256, 0, s->hi.stream>>>(a);
    const cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return sl_fail(s->h, SW_ECUDA, std::string("launch: ") + cudaGetErrorString(e));
    s->cur ^= 1;
    ++s->done;
  }
  return SW_OK;
}

extern "C" int sw_sl_end(sl_interval* s, const lm_result* out) {
  if (!s) return SW_EINVAL;
  if (!out) return sl_fail(s->h, SW_EINVAL, "out is NULL");
  if (s->done != s->p.n_steps) return sl_fail(s->h, SW_ESTATE, "the interval is not complete");
  double* dst[kMaxSL] = {};
  for (int k = 0; k < s->nf; ++k) {
    switch (s->bit[k]) {
      case LM_ZETA: dst[k] = out->zeta; break;
      case LM_H: dst[k] = out->h; break;
      case LM_U: dst[k] = out->u; break;
      case LM_V: dst[k] = out->v; break;
      default: dst[k] = out->q; break;
    }
  }
  const int N = s->hi.N;
  const long long np = (long long)N * N;
  const double T = (double)s->p.n_steps * s->hi.dt;
  cudaStream_t st = s->hi.stream;
  // results into the free buffers, then to the caller's pointers
  double* res = s->f[s->cur ^ 1];
  double* pos = s->d[s->cur ^ 1];
  k_sl_out<<<(unsigned)((np + 255) / 256), 256, 0, st>>>(s->g[s->cur], s->d[s->cur], res, pos, N, s->log2N, s->nf,
                                                         s->pos ? 1 : 0, T);
  cudaError_t e = cudaGetLastError();
  const cudaMemcpyKind kind = out->on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost;
  const size_t fb = (size_t)np * sizeof(double);
  for (int k = 0; k < s->nf && e == cudaSuccess; ++k)
    if (dst[k]) e = cudaMemcpyAsync(dst[k], res + k * np, fb, kind, st);
  if (s->pos && e == cudaSuccess && out->pos_x) e = cudaMemcpyAsync(out->pos_x, pos, fb, kind, st);
  if (s->pos && e == cudaSuccess && out->pos_y) e = cudaMemcpyAsync(out->pos_y, pos + np, fb, kind, st);
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  if (e != cudaSuccess) return sl_fail(s->h, SW_ECUDA, std::string("results: ") + cudaGetErrorString(e));
  sw_sl_destroy(s);
  return SW_OK;
}

extern "C" void sw_sl_destroy(sl_interval* s) {
  if (!s) return;
  if (s->arena) {
    cudaStreamSynchronize(s->hi.stream);
    cudaFree(s->arena);
  }
  delete s;
}
