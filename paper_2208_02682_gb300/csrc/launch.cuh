// launch.cuh -- host-side launchers for the kernels of kernels.cuh and
// stage.cuh.  Instantiated once per precision (kernels_f32.cu, kernels_f64.cu).
#pragma once
#include <string>

#include "stage.cuh"

struct sw_handle;

namespace lm {

// Rows per block of the row kernels: B rows of N points run with B*N/8
// threads (one 8-element Stockham butterfly set per thread and pass).
// `points` = B*N; 512 keeps small grids spread over many SMs.
inline int row_block_rows(int N, int points = 512) {
  // points = rows x N per block (the block runs points/8 threads per group)
  int B = points / N;
  if (B > N) B = N;
  if (B < 1) B = 1;
  return B;
}

// Row pass: B rows per block, W groups of N/8 threads per row (see
// k_stage_row_prod); the block may hold up to row_prod_max_threads threads.
template <typename T> size_t row_prod_smem(int N, int B, int W, const Layout& L) {
  const size_t nur = L.strategy == 2 ? 6 : 4, nug = (size_t)row_prod_group_rows(L);
  return (size_t)B * nur * N * sizeof(T) +
         (size_t)B * W * (2 * row_stride<T>(N) * sizeof(cplx<T>) + nug * N * sizeof(T));
}

// Largest W for B rows and npb product pairs per block: W > 1 needs whole
// warps per group (N >= 256), a thread count within the block limit, at most
// 15 named barriers (groups of N >= 512) and at most 110 KB of shared memory
// (two blocks per SM; one resident block per SM made the wider shape slower).
template <typename T> int row_prod_groups(int N, int B, int npb, const Layout& L) {
  const int strategy = L.strategy;
  const int G = N / 8;
  if (G < 32) return 1;
  int W = npb < 1 ? 1 : npb;
  while (W > 1 && (B * W * G > row_prod_max_threads<T>() || (G >= 64 && B * W > 15) ||
                   row_prod_smem<T>(N, B, W, L) > (size_t)110 * 1024))
    --W;
  // Strategy 2 transforms one base pair (xi) before the products, so the
  // row's other groups wait at the barrier; that pays only when every pair
  // gets a group of its own (measured slower at 1024^2 with 2 groups for 6
  // pairs)
  if (strategy == 2 && W < npb) W = 1;
  return W;
}

template <typename T> cudaError_t launch_col_inv(const ColInvArgs<T>& a, cudaStream_t s);
template <typename T> cudaError_t launch_col_fwd(const ColFwdArgs<T>& a, cudaStream_t s);
template <typename T, typename TO> cudaError_t launch_row_inv(const RowInvArgs<T, TO>& a, cudaStream_t s);
template <typename T> cudaError_t launch_row_fwd(const RowFwdArgs<T>& a, cudaStream_t s);
// warp: every run's rows have N <= 256 (groups of at most one warp), so the
// row kernels' variant without named barriers may run.  pdl: launch with
// programmatic stream serialisation (see pdl_wait).
template <typename T>
cudaError_t launch_stage(int kt, const RunDesc<T>* runs, const int* start, int nruns, int blocks, int threads,
                         size_t smem, int stage, bool warp, bool pdl, cudaStream_t s);
// Pipelined column forward pass of the large FP32 grids (L = log2 N in
// {10, 11}, four-column tiles): `blocks` persistent blocks over `total`
// work items.
cudaError_t launch_col_fwd_pipe(int L, const RunDesc<float>* runs, const int* start, int nruns, int blocks,
                                int threads, size_t smem, int total, bool pdl, cudaStream_t s);
// Resident blocks per SM of a pipelined column forward launch (0 on error).
int col_fwd_pipe_occupancy(int L, int threads, size_t smem);
template <typename T>
cudaError_t launch_spec_to_f64(const cplx<T>* y, const cplx<T>* comp, double2* out, long long ms, int fa, int fb,
                               double scale, cudaStream_t s);
template <typename T> cudaError_t launch_spec_from_f64(const double2* in, cplx<T>* y, long long n, cudaStream_t s);
template <typename T>
cudaError_t launch_velocity_from_vorticity(cplx<T>* y, const Geom& g, int fu, int fv, int fh, cudaStream_t s);
cudaError_t launch_diag(const double* phys, long long np, double f0, double c2, double* part, int nblk,
                        double* out, cudaStream_t s);
cudaError_t launch_add_real(double2* p, double delta, cudaStream_t s);
cudaError_t launch_spectrum_shells(const double2* F, int K, int KXP, double* acc, cudaStream_t s);

// Handle hooks for other translation units (defined in lagmean.cu).
struct HandleInfo {
  int N, model;
  double dt, f0, adv_x, adv_y;
  bool lm_open;
  cudaStream_t stream;
};
int handle_info(sw_handle* h, HandleInfo* hi);
// FP64 physical u, v, h, zeta of the state (4 * N * N doubles in the handle's
// staging buffer, valid until the handle's next call), on its stream
int handle_phys_uvhz(sw_handle* h, const double** out);
void handle_set_error(sw_handle* h, const std::string& msg);

#ifdef LM_INSTANTIATE
// Raise the dynamic shared-memory limit of every kernel once (outside any
// stream capture), to the device's opt-in maximum.
template <typename K> static cudaError_t allow_dynamic_smem(K kern, int optin) {
  // static and dynamic shared memory together may not exceed the opt-in limit
  cudaFuncAttributes fa;
  cudaError_t e = cudaFuncGetAttributes(&fa, kern);
  if (e != cudaSuccess) return e;
  return cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, optin - (int)fa.sharedSizeBytes);
}

template <typename T> static cudaError_t prepare_kernels_t() {
  int dev = 0, mx = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  if ((e = cudaDeviceGetAttribute(&mx, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev)) != cudaSuccess) return e;
  if ((e = allow_dynamic_smem(k_col_inv<T>, mx)) != cudaSuccess) return e;
  if ((e = allow_dynamic_smem(k_col_fwd<T>, mx)) != cudaSuccess) return e;
  if ((e = allow_dynamic_smem(k_row_inv<T, T>, mx)) != cudaSuccess) return e;
  if ((e = allow_dynamic_smem(k_row_fwd<T>, mx)) != cudaSuccess) return e;
  if ((e = allow_dynamic_smem(k_stage_col_inv<T>, mx)) != cudaSuccess) return e;
  if ((e = allow_dynamic_smem(k_stage_col_fwd<T>, mx)) != cudaSuccess) return e;
  if ((e = allow_dynamic_smem(k_stage_row_inv<T, false>, mx)) != cudaSuccess) return e;
  if ((e = allow_dynamic_smem(k_stage_row_inv<T, true>, mx)) != cudaSuccess) return e;
  if ((e = allow_dynamic_smem(k_stage_row_prod<T, false>, mx)) != cudaSuccess) return e;
  if ((e = allow_dynamic_smem(k_stage_row_prod<T, true>, mx)) != cudaSuccess) return e;
  return cudaSuccess;
}

template <typename T> cudaError_t launch_col_inv(const ColInvArgs<T>& a, cudaStream_t s) {
  const size_t sm = (size_t)4 * col_stride<T>(a.g.N, 4) * sizeof(cplx<T>);
  dim3 grid(a.g.KXP / 4, a.nout);
  k_col_inv<T><<<grid, a.g.N / 2, sm, s>>>(a);
  return cudaGetLastError();
}

template <typename T> cudaError_t launch_col_fwd(const ColFwdArgs<T>& a, cudaStream_t s) {
  const size_t sm = (size_t)4 * col_stride<T>(a.g.N, 4) * sizeof(cplx<T>);
  dim3 grid(a.g.KXP / 4, a.nout);
  k_col_fwd<T><<<grid, a.g.N / 2, sm, s>>>(a);
  return cudaGetLastError();
}

template <typename T, typename TO> cudaError_t launch_row_inv(const RowInvArgs<T, TO>& a, cudaStream_t s) {
  const size_t sm = (size_t)a.B * row_stride<T>(a.g.N) * sizeof(cplx<T>);
  k_row_inv<T, TO><<<a.g.N / a.B, a.B * a.g.N / 8, sm, s>>>(a);
  return cudaGetLastError();
}

template <typename T> cudaError_t launch_row_fwd(const RowFwdArgs<T>& a, cudaStream_t s) {
  const size_t sm = (size_t)a.B * row_stride<T>(a.g.N) * sizeof(cplx<T>);
  k_row_fwd<T><<<a.g.N / a.B, a.B * a.g.N / 8, sm, s>>>(a);
  return cudaGetLastError();
}

template <typename T>
cudaError_t launch_stage(int kt, const RunDesc<T>* runs, const int* start, int nruns, int blocks, int threads,
                         size_t smem, int stage, bool warp, bool pdl, cudaStream_t s) {
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3((unsigned)blocks);
  cfg.blockDim = dim3((unsigned)threads);
  cfg.dynamicSmemBytes = smem;
  cfg.stream = s;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  attr[0].val.programmaticStreamSerializationAllowed = 1;
  cfg.attrs = attr;
  cfg.numAttrs = pdl ? 1 : 0;
  switch (kt) {
    case KT_COL_INV: return cudaLaunchKernelEx(&cfg, k_stage_col_inv<T>, runs, start, nruns, stage);
    case KT_ROW_INV:
      return warp ? cudaLaunchKernelEx(&cfg, k_stage_row_inv<T, true>, runs, start, nruns)
                  : cudaLaunchKernelEx(&cfg, k_stage_row_inv<T, false>, runs, start, nruns);
    case KT_PHYS_Q: cfg.dynamicSmemBytes = 0; return cudaLaunchKernelEx(&cfg, k_stage_phys_q<T>, runs, start, nruns);
    case KT_ROW_PROD:
      return warp ? cudaLaunchKernelEx(&cfg, k_stage_row_prod<T, true>, runs, start, nruns, stage)
                  : cudaLaunchKernelEx(&cfg, k_stage_row_prod<T, false>, runs, start, nruns, stage);
    case KT_COL_FWD: return cudaLaunchKernelEx(&cfg, k_stage_col_fwd<T>, runs, start, nruns);
    default: cfg.dynamicSmemBytes = 0; return cudaLaunchKernelEx(&cfg, k_stage_update<T>, runs, start, nruns, stage);
  }
}

template <typename T>
cudaError_t launch_spec_to_f64(const cplx<T>* y, const cplx<T>* comp, double2* out, long long ms, int fa, int fb,
                               double scale, cudaStream_t s) {
  k_spec_to_f64<T><<<(unsigned)((ms + 255) / 256), 256, 0, s>>>(y, comp, out, ms, fa, fb, scale);
  return cudaGetLastError();
}

template <typename T> cudaError_t launch_spec_from_f64(const double2* in, cplx<T>* y, long long n, cudaStream_t s) {
  k_spec_from_f64<T><<<(unsigned)((n + 255) / 256), 256, 0, s>>>(in, y, n);
  return cudaGetLastError();
}

template <typename T>
cudaError_t launch_velocity_from_vorticity(cplx<T>* y, const Geom& g, int fu, int fv, int fh, cudaStream_t s) {
  k_velocity_from_vorticity<T><<<(unsigned)((g.ms + 255) / 256), 256, 0, s>>>(y, g, fu, fv, fh);
  return cudaGetLastError();
}

#define LM_INSTANTIATE_ALL(T)                                                                               \
  template cudaError_t launch_col_inv<T>(const ColInvArgs<T>&, cudaStream_t);                               \
  template cudaError_t launch_col_fwd<T>(const ColFwdArgs<T>&, cudaStream_t);                               \
  template cudaError_t launch_row_inv<T, T>(const RowInvArgs<T, T>&, cudaStream_t);                         \
  template cudaError_t launch_row_fwd<T>(const RowFwdArgs<T>&, cudaStream_t);                               \
  template cudaError_t launch_stage<T>(int, const RunDesc<T>*, const int*, int, int, int, size_t, int, bool,  \
                                       bool, cudaStream_t);                                                 \
  template cudaError_t launch_spec_to_f64<T>(const cplx<T>*, const cplx<T>*, double2*, long long, int, int,  \
                                             double, cudaStream_t);                                         \
  template cudaError_t launch_spec_from_f64<T>(const double2*, cplx<T>*, long long, cudaStream_t);            \
  template cudaError_t launch_velocity_from_vorticity<T>(cplx<T>*, const Geom&, int, int, int, cudaStream_t);
#endif

}  // namespace lm
