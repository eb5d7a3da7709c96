// remap.cu -- lmean_remap: Strategy-1 means onto the mean-position grid,
// Sec. 3.1, Eq. (remap-strat1), through the lift map Xi = (Xi^{-1})^{-1};
// lmean_lift: fields evaluated at given positions (the lift map of
// Strategy 2, Sec. 3.2), for the diagnostics of Secs. 4.2.1-4.2.2.
//
// One thread per grid point y = (x_i, y_j):
//   xi = 0; repeat iters times: xi <- d_I(y + xi),  d = x - Xi^{-1}(x)
//   fbar^L(y) = f~^L_I(y + xi)
// with d_I, f_I the periodic bilinear interpolants at a displacement from the
// grid point (cell i + floor(xi/dx), weight xi/dx - floor(xi/dx)).  Every
// operation is a separately rounded FP64 intrinsic, evaluated in the order
// written, so the results do not depend on the compiler's contraction choices.
#include <cuda_runtime.h>

#include <string>

#include "../../include/lagmean.h"

namespace lm {
void set_handleless_error(const std::string& msg);
}

namespace {

struct RemapArgs {
  const double* pos_x;
  const double* pos_y;
  const double* f[LM_REMAP_MAX_FIELDS];
  double* out[LM_REMAP_MAX_FIELDS];
  double* xi_x;
  double* xi_y;
  double* resid;
  int N, log2N, nf, iters;
};

// 2 pi in FP64 (twice the FP64 value of pi, exact)
constexpr double kTwoPi = 6.283185307179586476925286766559;

// grid coordinate x_i = (2 pi i) / N
__device__ __forceinline__ double coord(int i, int N) { return __ddiv_rn(__dmul_rn(kTwoPi, (double)i), (double)N); }

// bilinear weights and corner indices of a displacement (cx, cy) in cells
struct Cell {
  int i0, i1, j0, j1;
  double w00, w01, w10, w11;
};

__device__ __forceinline__ Cell cell_of(int i, int j, double cx, double cy, int N) {
  const double fx = floor(cx), fy = floor(cy);
  const double ax = __dsub_rn(cx, fx), ay = __dsub_rn(cy, fy);
  const unsigned msk = (unsigned)N - 1u;
  Cell c;
  c.i0 = (int)(((unsigned)i + (unsigned)(long long)fx) & msk);
  c.j0 = (int)(((unsigned)j + (unsigned)(long long)fy) & msk);
  c.i1 = (int)(((unsigned)c.i0 + 1u) & msk);
  c.j1 = (int)(((unsigned)c.j0 + 1u) & msk);
  const double bx = __dsub_rn(1.0, ax), by = __dsub_rn(1.0, ay);
  c.w00 = __dmul_rn(bx, by);
  c.w01 = __dmul_rn(ax, by);
  c.w10 = __dmul_rn(bx, ay);
  c.w11 = __dmul_rn(ax, ay);
  return c;
}

// w00 f00 + w01 f01 + w10 f10 + w11 f11, summed left to right
__device__ __forceinline__ double blend(const Cell& c, double f00, double f01, double f10, double f11) {
  double s = __dmul_rn(c.w00, f00);
  s = __dadd_rn(s, __dmul_rn(c.w01, f01));
  s = __dadd_rn(s, __dmul_rn(c.w10, f10));
  return __dadd_rn(s, __dmul_rn(c.w11, f11));
}

// Smem: the N grid coordinates (the same separately rounded values, computed
// once per block instead of four FP64 divisions per iteration).
__global__ void __launch_bounds__(256) k_remap(const __grid_constant__ RemapArgs a) {
  extern __shared__ double xs[];
  const int N = a.N;
  for (int t = threadIdx.x; t < N; t += blockDim.x) xs[t] = coord(t, N);
  __syncthreads();
  const long long np = (long long)N * N;
  const long long idx = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= np) return;
  const int i = (int)(idx & (N - 1)), j = (int)(idx >> a.log2N);
  const double inv_dx = __ddiv_rn((double)N, kTwoPi);
  double xx = 0.0, xy = 0.0, r = 0.0;
  for (int k = 0; k < a.iters; ++k) {
    const Cell c = cell_of(i, j, __dmul_rn(xx, inv_dx), __dmul_rn(xy, inv_dx), N);
    const long long o00 = (long long)c.j0 * N + c.i0, o01 = (long long)c.j0 * N + c.i1;
    const long long o10 = (long long)c.j1 * N + c.i0, o11 = (long long)c.j1 * N + c.i1;
    const double xi0 = xs[c.i0], xi1 = xs[c.i1];
    const double yj0 = xs[c.j0], yj1 = xs[c.j1];
    // d = x - Xi^{-1}(x) at the four corners
    const double nx = blend(c, __dsub_rn(xi0, a.pos_x[o00]), __dsub_rn(xi1, a.pos_x[o01]),
                            __dsub_rn(xi0, a.pos_x[o10]), __dsub_rn(xi1, a.pos_x[o11]));
    const double ny = blend(c, __dsub_rn(yj0, a.pos_y[o00]), __dsub_rn(yj0, a.pos_y[o01]),
                            __dsub_rn(yj1, a.pos_y[o10]), __dsub_rn(yj1, a.pos_y[o11]));
    if (k == a.iters - 1) r = fmax(fabs(__dsub_rn(nx, xx)), fabs(__dsub_rn(ny, xy)));
    xx = nx;
    xy = ny;
  }
  const Cell c = cell_of(i, j, __dmul_rn(xx, inv_dx), __dmul_rn(xy, inv_dx), N);
  const long long o00 = (long long)c.j0 * N + c.i0, o01 = (long long)c.j0 * N + c.i1;
  const long long o10 = (long long)c.j1 * N + c.i0, o11 = (long long)c.j1 * N + c.i1;
  for (int f = 0; f < a.nf; ++f) {
    const double* F = a.f[f];
    a.out[f][idx] = blend(c, F[o00], F[o01], F[o10], F[o11]);
  }
  if (a.xi_x) a.xi_x[idx] = __dadd_rn(xs[i], xx);
  if (a.xi_y) a.xi_y[idx] = __dadd_rn(xs[j], xy);
  if (a.resid) a.resid[idx] = r;
}

struct LiftArgs {
  const double* pos_x;
  const double* pos_y;
  const double* f[LM_REMAP_MAX_FIELDS];
  double* out[LM_REMAP_MAX_FIELDS];
  int N, log2N, nf;
};

// out(y) = f_I(pos(y)), the displacement pos - y taken from the grid point
// (same rounding steps as the remap's final interpolation)
__global__ void __launch_bounds__(256) k_lift(const __grid_constant__ LiftArgs a) {
  extern __shared__ double xs[];
  const int N = a.N;
  for (int t = threadIdx.x; t < N; t += blockDim.x) xs[t] = coord(t, N);
  __syncthreads();
  const long long np = (long long)N * N;
  const long long idx = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= np) return;
  const int i = (int)(idx & (N - 1)), j = (int)(idx >> a.log2N);
  const double inv_dx = __ddiv_rn((double)N, kTwoPi);
  const double xx = __dsub_rn(a.pos_x[idx], xs[i]), xy = __dsub_rn(a.pos_y[idx], xs[j]);
  const Cell c = cell_of(i, j, __dmul_rn(xx, inv_dx), __dmul_rn(xy, inv_dx), N);
  const long long o00 = (long long)c.j0 * N + c.i0, o01 = (long long)c.j0 * N + c.i1;
  const long long o10 = (long long)c.j1 * N + c.i0, o11 = (long long)c.j1 * N + c.i1;
  for (int f = 0; f < a.nf; ++f) {
    const double* F = a.f[f];
    a.out[f][idx] = blend(c, F[o00], F[o01], F[o10], F[o11]);
  }
}

int fail(const std::string& m, int rc) {
  lm::set_handleless_error("lmean_remap: " + m);
  return rc;
}

int fail_lift(const std::string& m, int rc) {
  lm::set_handleless_error("lmean_lift: " + m);
  return rc;
}

}  // namespace

extern "C" int lmean_remap(int N, const double* pos_x, const double* pos_y, int nfields,
                           const double* const* ftilde, double* const* fbar, int iters, double* xi_x, double* xi_y,
                           double* resid, void* stream) {
  if (N < 16 || N > 4096 || (N & (N - 1)) != 0) return fail("N must be a power of two in [16, 4096]", SW_EINVAL);
  if (!pos_x || !pos_y) return fail("pos_x and pos_y are required", SW_EINVAL);
  if (nfields < 0 || nfields > LM_REMAP_MAX_FIELDS)
    return fail("nfields must be in [0, " + std::to_string(LM_REMAP_MAX_FIELDS) + "]", SW_EINVAL);
  if (nfields > 0 && (!ftilde || !fbar)) return fail("ftilde and fbar arrays are required", SW_EINVAL);
  if (iters < 1 || iters > 10000) return fail("iters must be in [1, 10000]", SW_EINVAL);
  RemapArgs a = {};
  a.pos_x = pos_x;
  a.pos_y = pos_y;
  a.N = N;
  a.log2N = 0;
  while ((1 << a.log2N) < N) ++a.log2N;
  a.nf = nfields;
  a.iters = iters;
  a.xi_x = xi_x;
  a.xi_y = xi_y;
  a.resid = resid;
  const void* ins[2 + LM_REMAP_MAX_FIELDS];
  int nin = 0;
  ins[nin++] = pos_x;
  ins[nin++] = pos_y;
  for (int f = 0; f < nfields; ++f) {
    if (!ftilde[f] || !fbar[f]) return fail("null field pointer", SW_EINVAL);
    a.f[f] = ftilde[f];
    a.out[f] = fbar[f];
    ins[nin++] = ftilde[f];
  }
  // outputs are written while neighbouring points are still being gathered
  const void* outs[3 + LM_REMAP_MAX_FIELDS];
  int nout = 0;
  for (int f = 0; f < nfields; ++f) outs[nout++] = fbar[f];
  if (xi_x) outs[nout++] = xi_x;
  if (xi_y) outs[nout++] = xi_y;
  if (resid) outs[nout++] = resid;
  for (int p = 0; p < nout; ++p) {
    for (int q = 0; q < nin; ++q)
      if (outs[p] == ins[q]) return fail("an output aliases an input", SW_EINVAL);
    for (int q = p + 1; q < nout; ++q)
      if (outs[p] == outs[q]) return fail("two outputs share a buffer", SW_EINVAL);
  }
  const long long np = (long long)N * N;
  const unsigned blocks = (unsigned)((np + 255) / 256);
  k_remap<<<blocks, 256, (size_t)N * sizeof(double), (cudaStream_t)stream>>>(a);
  const cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return fail(std::string("launch: ") + cudaGetErrorString(e), SW_ECUDA);
  return SW_OK;
}

extern "C" int lmean_lift(int N, const double* pos_x, const double* pos_y, int nfields, const double* const* f,
                          double* const* out, void* stream) {
  if (N < 16 || N > 4096 || (N & (N - 1)) != 0) return fail_lift("N must be a power of two in [16, 4096]", SW_EINVAL);
  if (!pos_x || !pos_y) return fail_lift("pos_x and pos_y are required", SW_EINVAL);
  if (nfields < 1 || nfields > LM_REMAP_MAX_FIELDS)
    return fail_lift("nfields must be in [1, " + std::to_string(LM_REMAP_MAX_FIELDS) + "]", SW_EINVAL);
  if (!f || !out) return fail_lift("f and out arrays are required", SW_EINVAL);
  LiftArgs a = {};
  a.pos_x = pos_x;
  a.pos_y = pos_y;
  a.N = N;
  while ((1 << a.log2N) < N) ++a.log2N;
  a.nf = nfields;
  for (int k = 0; k < nfields; ++k) {
    if (!f[k] || !out[k]) return fail_lift("null field pointer", SW_EINVAL);
    a.f[k] = f[k];
    a.out[k] = out[k];
  }
  // an output may not be an input (neighbouring points are gathered while
  // outputs are written) nor another output
  for (int k = 0; k < nfields; ++k) {
    if (out[k] == pos_x || out[k] == pos_y) return fail_lift("an output aliases an input", SW_EINVAL);
    for (int m = 0; m < nfields; ++m)
      if (out[k] == f[m] || (m > k && out[k] == out[m])) return fail_lift("an output aliases another buffer", SW_EINVAL);
  }
  const long long np = (long long)N * N;
  k_lift<<<(unsigned)((np + 255) / 256), 256, (size_t)N * sizeof(double), (cudaStream_t)stream>>>(a);
  const cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return fail_lift(std::string("launch: ") + cudaGetErrorString(e), SW_ECUDA);
  return SW_OK;
}
