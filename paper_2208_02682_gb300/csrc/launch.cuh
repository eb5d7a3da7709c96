// launch.cuh -- host-side launchers for the kernels of kernels.cuh.
// Instantiated once per precision (kernels_f32.cu, kernels_f64.cu).
#pragma once
#include "kernels.cuh"

namespace lm {

// Rows per block of the row kernels: B rows of N points run with B*N/8
// threads (one 8-element Stockham butterfly set per thread and pass).
// `points` = B*N; 512 keeps small grids spread over many SMs.
inline int row_block_rows(int N, int points = 512) {
  int B = points / N;
  if (B > N) B = N;
  if (B < 1) B = 1;
  return B;
}

template <typename T> size_t row_prod_smem(int N, int B, int strategy) {
  return (size_t)2 * B * pad8(N) * sizeof(cplx<T>) + (size_t)(strategy == 2 ? 6 : 4) * B * N * sizeof(T);
}

template <typename T> cudaError_t launch_col_inv(const ColInvArgs<T>& a, cudaStream_t s);
template <typename T> cudaError_t launch_col_fwd(const ColFwdArgs<T>& a, cudaStream_t s);
template <typename T, typename TO> cudaError_t launch_row_inv(const RowInvArgs<T, TO>& a, cudaStream_t s);
template <typename T> cudaError_t launch_row_fwd(const RowFwdArgs<T>& a, cudaStream_t s);
template <typename T> cudaError_t launch_row_prod(const RowProdArgs<T>& a, cudaStream_t s);
template <typename T> cudaError_t launch_update(const UpdateArgs<T>& a, cudaStream_t s);
template <typename T> cudaError_t launch_phys_q(T* phys, long long np, double f0, cudaStream_t s);
template <typename T>
cudaError_t launch_spec_to_f64(const cplx<T>* y, const cplx<T>* comp, double2* out, long long ms, int fa, int fb,
                               double scale, cudaStream_t s);
template <typename T> cudaError_t launch_spec_from_f64(const double2* in, cplx<T>* y, long long n, cudaStream_t s);
cudaError_t launch_diag(const double* phys, long long np, double f0, double c2, double* part, int nblk,
                        double* out, cudaStream_t s);

#ifdef LM_INSTANTIATE
// Raise the dynamic shared-memory limit of every kernel once (outside any
// stream capture), to the device's opt-in maximum.
template <typename T> static cudaError_t prepare_kernels_t() {
  int dev = 0, mx = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  if ((e = cudaDeviceGetAttribute(&mx, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev)) != cudaSuccess) return e;
  const cudaFuncAttribute A = cudaFuncAttributeMaxDynamicSharedMemorySize;
  if ((e = cudaFuncSetAttribute(k_col_inv<T>, A, mx)) != cudaSuccess) return e;
  if ((e = cudaFuncSetAttribute(k_col_fwd<T>, A, mx)) != cudaSuccess) return e;
  if ((e = cudaFuncSetAttribute(k_row_inv<T, T>, A, mx)) != cudaSuccess) return e;
  if ((e = cudaFuncSetAttribute(k_row_fwd<T>, A, mx)) != cudaSuccess) return e;
  if ((e = cudaFuncSetAttribute(k_row_prod<T>, A, mx)) != cudaSuccess) return e;
  return cudaSuccess;
}

template <typename T> cudaError_t launch_col_inv(const ColInvArgs<T>& a, cudaStream_t s) {
  const size_t sm = (size_t)4 * pad8(a.g.N) * sizeof(cplx<T>);
  dim3 grid(a.g.KXP / 4, a.nout);
  k_col_inv<T><<<grid, a.g.N / 2, sm, s>>>(a);
  return cudaGetLastError();
}

template <typename T> cudaError_t launch_col_fwd(const ColFwdArgs<T>& a, cudaStream_t s) {
  const size_t sm = (size_t)4 * pad8(a.g.N) * sizeof(cplx<T>);
  dim3 grid(a.g.KXP / 4, a.nout);
  k_col_fwd<T><<<grid, a.g.N / 2, sm, s>>>(a);
  return cudaGetLastError();
}

template <typename T, typename TO> cudaError_t launch_row_inv(const RowInvArgs<T, TO>& a, cudaStream_t s) {
  const size_t sm = (size_t)a.B * pad8(a.g.N) * sizeof(cplx<T>);
  k_row_inv<T, TO><<<a.g.N / a.B, a.B * a.g.N / 8, sm, s>>>(a);
  return cudaGetLastError();
}

template <typename T> cudaError_t launch_row_fwd(const RowFwdArgs<T>& a, cudaStream_t s) {
  const size_t sm = (size_t)a.B * pad8(a.g.N) * sizeof(cplx<T>);
  k_row_fwd<T><<<a.g.N / a.B, a.B * a.g.N / 8, sm, s>>>(a);
  return cudaGetLastError();
}

template <typename T> cudaError_t launch_row_prod(const RowProdArgs<T>& a, cudaStream_t s) {
  const size_t sm = row_prod_smem<T>(a.g.N, a.B, a.L.strategy);
  const int npairs = (a.L.np + 1) / 2;
  dim3 grid(a.g.N / a.B, (npairs + a.ppb - 1) / a.ppb);
  k_row_prod<T><<<grid, a.B * a.g.N / 8, sm, s>>>(a);
  return cudaGetLastError();
}

template <typename T> cudaError_t launch_update(const UpdateArgs<T>& a, cudaStream_t s) {
  const int thr = 256;
  const long long nb = (a.g.ms + thr - 1) / thr;
  k_update<T><<<dim3((unsigned)nb, a.L.nf), thr, 0, s>>>(a);
  return cudaGetLastError();
}

template <typename T> cudaError_t launch_phys_q(T* phys, long long np, double f0, cudaStream_t s) {
  k_phys_q<T><<<(unsigned)((np + 255) / 256), 256, 0, s>>>(phys, np, f0);
  return cudaGetLastError();
}

template <typename T>
cudaError_t launch_spec_to_f64(const cplx<T>* y, const cplx<T>* comp, double2* out, long long ms, int fa, int fb,
                               double scale, cudaStream_t s) {
  k_spec_to_f64<T><<<(unsigned)((ms + 255) / 256), 256, 0, s>>>(y, comp, out, ms, 0, nullptr, fa, fb, scale);
  return cudaGetLastError();
}

template <typename T> cudaError_t launch_spec_from_f64(const double2* in, cplx<T>* y, long long n, cudaStream_t s) {
  k_spec_from_f64<T><<<(unsigned)((n + 255) / 256), 256, 0, s>>>(in, y, n);
  return cudaGetLastError();
}

#define LM_INSTANTIATE_ALL(T)                                                                             \
  template cudaError_t launch_col_inv<T>(const ColInvArgs<T>&, cudaStream_t);                             \
  template cudaError_t launch_col_fwd<T>(const ColFwdArgs<T>&, cudaStream_t);                             \
  template cudaError_t launch_row_inv<T, T>(const RowInvArgs<T, T>&, cudaStream_t);                       \
  template cudaError_t launch_row_fwd<T>(const RowFwdArgs<T>&, cudaStream_t);                             \
  template cudaError_t launch_row_prod<T>(const RowProdArgs<T>&, cudaStream_t);                           \
  template cudaError_t launch_update<T>(const UpdateArgs<T>&, cudaStream_t);                              \
  template cudaError_t launch_phys_q<T>(T*, long long, double, cudaStream_t);                             \
  template cudaError_t launch_spec_to_f64<T>(const cplx<T>*, const cplx<T>*, double2*, long long, int, int, \
                                             double, cudaStream_t);                                       \
  template cudaError_t launch_spec_from_f64<T>(const double2*, cplx<T>*, long long, cudaStream_t);
#endif

}  // namespace lm
