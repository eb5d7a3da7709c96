// FP64 instantiation of the stage kernels and their launchers, plus the FP64
// invariant reductions.
#define LM_INSTANTIATE
#include "launch.cuh"

namespace lm {
LM_INSTANTIATE_ALL(double)
cudaError_t prepare_kernels_f64() { return prepare_kernels_t<double>(); }

// Energy density h |u|^2/2 + c2 h^2/2 and potential enstrophy h q^2/2 with
// q = (f0 + zeta)/h, summed per block with a fixed tree.
__global__ void __launch_bounds__(256) k_diag_partial(const double* __restrict__ phys, long long np, double f0,
                                                      double c2, double* __restrict__ part) {
  __shared__ double se[256], sz[256];
  double e = 0.0, z = 0.0;
  const long long stride = (long long)gridDim.x * blockDim.x;
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < np; i += stride) {
    const double u = phys[i], v = phys[np + i], h = phys[2 * np + i], zeta = phys[3 * np + i];
    const double q = (f0 + zeta) / h;
    e += 0.5 * h * (u * u + v * v) + 0.5 * c2 * h * h;
    z += 0.5 * h * q * q;
  }
  se[threadIdx.x] = e;
  sz[threadIdx.x] = z;
  __syncthreads();
  for (int w = 128; w > 0; w >>= 1) {
    if (threadIdx.x < w) {
      se[threadIdx.x] += se[threadIdx.x + w];
      sz[threadIdx.x] += sz[threadIdx.x + w];
    }
    __syncthreads();
  }
  if (threadIdx.x == 0) {
    part[2 * blockIdx.x] = se[0];
    part[2 * blockIdx.x + 1] = sz[0];
  }
}

__global__ void __launch_bounds__(256) k_diag_final(const double* __restrict__ part, int nblk, long long np,
                                                    double* __restrict__ out) {
  __shared__ double se[256], sz[256];
  double e = 0.0, z = 0.0;
  for (int i = threadIdx.x; i < nblk; i += blockDim.x) {
    e += part[2 * i];
    z += part[2 * i + 1];
  }
  se[threadIdx.x] = e;
  sz[threadIdx.x] = z;
  __syncthreads();
  for (int w = 128; w > 0; w >>= 1) {
    if (threadIdx.x < w) {
      se[threadIdx.x] += se[threadIdx.x + w];
      sz[threadIdx.x] += sz[threadIdx.x + w];
    }
    __syncthreads();
  }
  if (threadIdx.x == 0) {
    out[1] = se[0] / (double)np;
    out[2] = sz[0] / (double)np;
  }
}

__global__ void k_add_real(double2* p, double delta) {
  if (threadIdx.x == 0 && blockIdx.x == 0) p->x += delta;
}

// Shell sums of |F|^2/2 over the whole plane from the kx >= 0 half of the
// 2/3 box (FP64 spectral layout [ky + K][kx], row stride KXP): shell
// round(|k|), weight 2 for kx > 0 (the mirrored half).
__global__ void k_spectrum_shells(const double2* __restrict__ F, int K, int KXP, double* __restrict__ acc) {
  const int NY = 2 * K + 1;
  const long long m = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (m >= (long long)NY * KXP) return;
  const int kyi = (int)(m / KXP), kx = (int)(m - (long long)kyi * KXP);
  if (kx > K) return;
  const int ky = kyi - K;
  const int sh = (int)floor(sqrt((double)(kx * kx + ky * ky)) + 0.5);
  const double2 v = F[m];
  atomicAdd(acc + sh, (kx == 0 ? 0.5 : 1.0) * (v.x * v.x + v.y * v.y));
}

cudaError_t launch_spectrum_shells(const double2* F, int K, int KXP, double* acc, cudaStream_t s) {
  const long long n = (long long)(2 * K + 1) * KXP;
  k_spectrum_shells<<<(unsigned)((n + 255) / 256), 256, 0, s>>>(F, K, KXP, acc);
  return cudaGetLastError();
}

cudaError_t launch_add_real(double2* p, double delta, cudaStream_t s) {
  k_add_real<<<1, 1, 0, s>>>(p, delta);
  return cudaGetLastError();
}

cudaError_t launch_diag(const double* phys, long long np, double f0, double c2, double* part, int nblk,
                        double* out, cudaStream_t s) {
  k_diag_partial<<<nblk, 256, 0, s>>>(phys, np, f0, c2, part);
  k_diag_final<<<1, 256, 0, s>>>(part, nblk, np, out);
  return cudaGetLastError();
}
}  // namespace lm
