// fft.cuh -- block-wide power-of-two complex FFTs in shared memory.
//
// Stockham autosort formulation (natural-order input and output, no bit
// reversal): pass p with stride Ns = R_0 R_1 ... R_{p-1} and radix R maps,
// for every j in [0, N/R) with k = j mod Ns,
//   v_r = x[j + r N/R] * w^{r k},  w = exp(sigma 2 pi i / (Ns R)),
//   y[(j - k) R + k + q Ns] = sum_r v_r exp(sigma 2 pi i r q / R).
// Radix-8 passes first, then one radix-4 or radix-2 pass for the remaining
// bits.  Each thread owns exactly 8 elements per pass (one radix-8 butterfly,
// two radix-4 or four radix-2 butterflies), so a block of B transforms of
// length N runs with B*N/8 threads.  The pass reads all of its elements into
// registers, synchronises, then writes in place.
//
// Transform b lives at buf + b*bstride, element n at pad8(n).  The twiddle
// table holds tw[t] = exp(-2 pi i t / N), t < N (computed in FP64 on the host
// and rounded to T); the inverse transform (sigma = +1) uses its conjugate.
// No normalisation is applied.
#pragma once
#include "common.cuh"

namespace lm {

template <typename T, int SIGN>
__device__ __forceinline__ cplx<T> mul_sigma_i(cplx<T> a) {  // a * (sigma i)
  return SIGN > 0 ? mk<T>(-a.y, a.x) : mk<T>(a.y, -a.x);
}

template <typename T, int SIGN>
__device__ __forceinline__ void dft4(cplx<T>& a0, cplx<T>& a1, cplx<T>& a2, cplx<T>& a3) {
  cplx<T> t0 = cadd<T>(a0, a2), t1 = csub<T>(a0, a2);
  cplx<T> t2 = cadd<T>(a1, a3), t3 = mul_sigma_i<T, SIGN>(csub<T>(a1, a3));
  a0 = cadd<T>(t0, t2);
  a2 = csub<T>(t0, t2);
  a1 = cadd<T>(t1, t3);
  a3 = csub<T>(t1, t3);
}

template <typename T, int SIGN>
__device__ __forceinline__ void dft8(cplx<T>* v) {
  cplx<T> a0 = v[0], a1 = v[2], a2 = v[4], a3 = v[6];
  cplx<T> b0 = v[1], b1 = v[3], b2 = v[5], b3 = v[7];
  dft4<T, SIGN>(a0, a1, a2, a3);
  dft4<T, SIGN>(b0, b1, b2, b3);
  const T h = (T)0.70710678118654752440;
  // b_q *= exp(sigma 2 pi i q / 8)
  b1 = mk<T>((b1.x - SIGN * b1.y) * h, (SIGN * b1.x + b1.y) * h);
  b2 = mul_sigma_i<T, SIGN>(b2);
  b3 = mk<T>((-b3.x - SIGN * b3.y) * h, (SIGN * b3.x - b3.y) * h);
  v[0] = cadd<T>(a0, b0); v[4] = csub<T>(a0, b0);
  v[1] = cadd<T>(a1, b1); v[5] = csub<T>(a1, b1);
  v[2] = cadd<T>(a2, b2); v[6] = csub<T>(a2, b2);
  v[3] = cadd<T>(a3, b3); v[7] = csub<T>(a3, b3);
}

// Twiddle exp(sigma 2 pi i e 2^tstep / N).  From the table (host FP64
// values rounded to T), or, with TWC and FP32, from sincospif: that removes
// the scattered table loads of the late passes, whose L1 wavefronts limit
// kernels with many resident warps (the column passes); kernels with few
// resident warps (the row passes) hide table loads better than the longer
// sincospif chain.  The argument e 2^(tstep+1-log2N) is exact in FP32.
template <typename T, int SIGN, bool TWC>
__device__ __forceinline__ cplx<T> twiddle(int e, int tstep, int log2N, const cplx<T>* __restrict__ tw) {
  cplx<T> t;
  if (TWC && sizeof(T) == 4) {
    float s, c;
    sincospif(ldexpf((float)e, tstep + 1 - log2N), &s, &c);
    t.x = (T)c;
    t.y = (T)(-s);
  } else {
    t = __ldg(&tw[e << tstep]);
  }
  if (SIGN > 0) t.y = -t.y;
  return t;
}

// Twiddles w^{r k}, r < R, of one butterfly from three evaluations (w^k,
// w^2k, w^4k); the others are products of those (at most two
// multiplications deep).
template <typename T, int SIGN, int R, bool TWC>
__device__ __forceinline__ void butterfly_twiddles(cplx<T>* w, int k, int tstep, int log2N,
                                                   const cplx<T>* __restrict__ tw) {
  auto ld = [&](int e) { return twiddle<T, SIGN, TWC>(e, tstep, log2N, tw); };
  w[1] = ld(k);
  if (R >= 4) {
    w[2] = ld(2 * k);
    w[3] = cmul<T>(w[1], w[2]);
  }
  if (R == 8) {
    w[4] = ld(4 * k);
    w[5] = cmul<T>(w[4], w[1]);
    w[6] = cmul<T>(w[4], w[2]);
    w[7] = cmul<T>(w[4], w[3]);
  }
}

template <typename T, int SIGN, int LR, bool TWC>
__device__ __forceinline__ void stockham_pass(cplx<T>* buf, int log2N, int lNs, int bstride,
                                              const cplx<T>* __restrict__ tw) {
  constexpr int R = 1 << LR;
  constexpr int NB = 8 / R;  // butterflies per thread
  const int lNR = log2N - LR;
  const int NR = 1 << lNR;
  const int Ns = 1 << lNs;
  const int tstep = log2N - lNs - LR;  // table index = (r*k) << tstep
  const int nthr = blockDim.x;
  cplx<T> v[8];
  int base[NB], outb[NB];
#pragma unroll
  for (int u = 0; u < NB; ++u) {
    const int g = u * nthr + threadIdx.x;
    const int b = g >> lNR;
    const int j = g & (NR - 1);
    const int k = j & (Ns - 1);
    const cplx<T>* src = buf + b * bstride;
    base[u] = b * bstride;
    outb[u] = ((j - k) << LR) + k;
#pragma unroll
    for (int r = 0; r < R; ++r) v[u * R + r] = src[pad8(j + r * NR)];
    if (k > 0) {
      cplx<T> w[R];
      butterfly_twiddles<T, SIGN, R, TWC>(w, k, tstep, log2N, tw);
#pragma unroll
      for (int r = 1; r < R; ++r) v[u * R + r] = cmul<T>(v[u * R + r], w[r]);
    }
  }
  __syncthreads();
#pragma unroll
  for (int u = 0; u < NB; ++u) {
    cplx<T>* vv = v + u * R;
    if (LR == 3) {
      dft8<T, SIGN>(vv);
    } else if (LR == 2) {
      dft4<T, SIGN>(vv[0], vv[1], vv[2], vv[3]);
    } else {
      cplx<T> a = vv[0], b = vv[1];
      vv[0] = cadd<T>(a, b);
      vv[1] = csub<T>(a, b);
    }
#pragma unroll
    for (int q = 0; q < R; ++q) buf[base[u] + pad8(outb[u] + q * Ns)] = vv[q];
  }
  __syncthreads();
}

// Block-wide FFT of `batch` transforms of length 2^log2N; requires
// blockDim.x * 8 == batch * 2^log2N and log2N >= 1.  Callers synchronise
// before (data in place); the function ends with a barrier.  TWC: computed
// FP32 twiddles (see twiddle()).
template <typename T, int SIGN, bool TWC = false>
__device__ void block_fft(cplx<T>* buf, int log2N, int bstride, const cplx<T>* __restrict__ tw) {
  int lNs = 0;
  int rem = log2N;
  while (rem >= 3) {
    stockham_pass<T, SIGN, 3, TWC>(buf, log2N, lNs, bstride, tw);
    lNs += 3;
    rem -= 3;
  }
  if (rem == 2) stockham_pass<T, SIGN, 2, TWC>(buf, log2N, lNs, bstride, tw);
  if (rem == 1) stockham_pass<T, SIGN, 1, TWC>(buf, log2N, lNs, bstride, tw);
}

}  // namespace lm
