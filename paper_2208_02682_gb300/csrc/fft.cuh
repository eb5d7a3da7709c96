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
// Transform b lives at buf + b*bstride, element n at sidx<T>(n).  Twiddles come
// from a pass-ordered table: the pass with stride Ns and radix R reads
//   tw[r*Ns + k - 1] = exp(-2 pi i r k / (Ns R)),  1 <= r < R, 0 <= k < Ns,
// (rows r of Ns consecutive entries; the index ranges of successive passes
// tile [0, N-1)), so a warp's loads for one r are contiguous.  The table is
// computed in FP64 on the host (fft_twiddle_table) and rounded to T; the
// inverse transform (sigma = +1) uses its conjugate.  No normalisation.
#pragma once
#include <cmath>
#include <vector>

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

// Pass sequence shared by the kernels (block_fft, gfft) and the host
// table builder: radix-8 passes, then one radix-4 or radix-2 pass for the
// remaining bits.
__host__ __device__ __forceinline__ int fft_num_passes(int log2N) { return (log2N + 2) / 3; }
__host__ __device__ __forceinline__ int fft_pass_lr(int log2N, int p) {
  return p < log2N / 3 ? 3 : log2N % 3;
}

// Twiddles w^{r k}, 1 <= r < R, w = exp(sigma 2 pi i / (Ns R)), of one
// butterfly.  FP64 loads all R - 1 from the table (FP64 multiplies are the
// scarce resource).  FP32 evaluates w^k, w^2k, w^4k and forms the others as
// products (at most two multiplications deep): from the table rows r = 1, 2,
// 4, or, with TWC, from sincospif of 2 e / (Ns R) (exact in FP32) for e = k,
// 2k, 4k.  The generic column kernels compute them; the stage kernels load
// the table (their loads stay in L1; at 1024^2-2048^2 the column passes ran
// 10-15% faster with the table than with sincospif).
template <typename T, int SIGN, int R, bool TWC>
__device__ __forceinline__ void butterfly_twiddles(cplx<T>* w, int k, int lNs, const cplx<T>* __restrict__ tw) {
  constexpr int LR = R == 8 ? 3 : (R == 4 ? 2 : 1);
  const cplx<T>* t = tw + (k - 1);
  if (sizeof(T) == 4) {
    auto ev = [&](int r) {
      cplx<T> c;
      if (TWC) {
        float sn, cs;
        sincospif(ldexpf((float)(r * k), 1 - lNs - LR), &sn, &cs);
        c.x = (T)cs;
        c.y = (T)(-sn);
      } else {
        c = __ldg(t + (r << lNs));
      }
      if (SIGN > 0) c.y = -c.y;
      return c;
    };
    w[1] = ev(1);
    if (R >= 4) {
      w[2] = ev(2);
      w[3] = cmul<T>(w[1], w[2]);
    }
    if (R == 8) {
      w[4] = ev(4);
      w[5] = cmul<T>(w[4], w[1]);
      w[6] = cmul<T>(w[4], w[2]);
      w[7] = cmul<T>(w[4], w[3]);
    }
  } else {
#pragma unroll
    for (int r = 1; r < R; ++r) {
      w[r] = __ldg(t + (r << lNs));
      if (SIGN > 0) w[r].y = -w[r].y;
    }
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
    for (int r = 0; r < R; ++r) v[u * R + r] = src[sidx<T>(j + r * NR)];
    if (k > 0) {
      cplx<T> w[R];
      butterfly_twiddles<T, SIGN, R, TWC>(w, k, lNs, tw);
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
    for (int q = 0; q < R; ++q) buf[base[u] + sidx<T>(outb[u] + q * Ns)] = vv[q];
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

template <typename T, int SIGN, int R>
__device__ __forceinline__ void dft_r(cplx<T>* v) {
  if (R == 8) {
    dft8<T, SIGN>(v);
  } else if (R == 4) {
    dft4<T, SIGN>(v[0], v[1], v[2], v[3]);
  } else {
    const cplx<T> a = v[0], b = v[1];
    v[0] = cadd<T>(a, b);
    v[1] = csub<T>(a, b);
  }
}

// ---------------------------------------------------------------------------
// Register-resident transforms owned by a group of G = N/8 threads (one
// transform per group; groups never wait for one another), N = 2^L fixed at
// compile time.  Thread j of the group holds elements j + m G, m < 8, of its
// transform in x[m] on entry (input) and on exit (output): the first pass's
// butterflies read exactly these positions, and the last pass's butterflies
// write them.  The passes in between exchange through two shared buffers
// used alternately, so each pass costs one group barrier.  Every stride,
// shared-memory offset and twiddle-table offset is a compile-time constant
// (with run-time lengths the index arithmetic cost more instructions than
// the butterflies), and twiddles are applied without a branch at k = 0 (the
// table holds w^0 = 1 there; the product is exact).
// SYNC: 0 the warp (G <= 32: several groups per warp execute the same
// instructions), 1 named barrier grp + 1 over the group's G threads, 2 the
// block (groups whose threads interleave, column tiles).  A named barrier
// with a run-time id reserves all 16 of a block's barriers, which limits the
// blocks resident on an SM, so kernels whose groups all fit in a warp are
// compiled without it.

template <int SYNC, int G>
__device__ __forceinline__ void gsync(int grp) {
  if (SYNC == 2) __syncthreads();
  else if (SYNC == 1) asm volatile("bar.sync %0, %1;" ::"r"(grp + 1), "r"(G) : "memory");
  else __syncwarp();
}

// Twiddles w^{r k}, 1 <= r < R, of a butterfly of the pass with stride
// Ns = 2^LNS (see butterfly_twiddles).
template <typename T, int SIGN, int R, int LNS, bool TWC>
__device__ __forceinline__ void twiddles_ct(cplx<T>* w, int k, const cplx<T>* __restrict__ tw) {
  constexpr int LR = R == 8 ? 3 : (R == 4 ? 2 : 1);
  const cplx<T>* t = tw + (k - 1);
  if (sizeof(T) == 4) {
    auto ev = [&](int r) {
      cplx<T> c;
      if (TWC) {
        float sn, cs;
        // 2 r k / (Ns R), exact in FP32 (a power-of-two scale)
        sincospif((float)(r * k) * (2.0f / (float)(1 << (LNS + LR))), &sn, &cs);
        c.x = (T)cs;
        c.y = (T)(-sn);
      } else {
        c = __ldg(t + (r << LNS));
      }
      if (SIGN > 0) c.y = -c.y;
      return c;
    };
    w[1] = ev(1);
    if (R >= 4) {
      w[2] = ev(2);
      w[3] = cmul<T>(w[1], w[2]);
    }
    if (R == 8) {
      w[4] = ev(4);
      w[5] = cmul<T>(w[4], w[1]);
      w[6] = cmul<T>(w[4], w[2]);
      w[7] = cmul<T>(w[4], w[3]);
    }
  } else {
#pragma unroll
    for (int r = 1; r < R; ++r) {
      w[r] = __ldg(t + (r << LNS));
      if (SIGN > 0) w[r].y = -w[r].y;
    }
  }
}

// Middle pass P (radix 8, stride Ns = 8^P) from `in` to `out`.
template <typename T, int SIGN, int L, int P, bool TWC>
__device__ __forceinline__ void gpass8(const cplx<T>* in, cplx<T>* out, int j, const cplx<T>* __restrict__ tw) {
  constexpr int G = 1 << (L - 3), LNS = 3 * P, NS = 1 << LNS;
  constexpr int RS = G + G / 8;    // shared-memory distance of G positions (G % 8 == 0)
  constexpr int WS = NS + NS / 8;  // of Ns positions
  cplx<T> v[8];
  const int rb = j + (j >> 3);
#pragma unroll
  for (int r = 0; r < 8; ++r) v[r] = in[rb + r * RS];
  const int k = j & (NS - 1);
  cplx<T> wr[8];
  twiddles_ct<T, SIGN, 8, LNS, TWC>(wr, k, tw);
#pragma unroll
  for (int r = 1; r < 8; ++r) v[r] = cmul<T>(v[r], wr[r]);
  dft8<T, SIGN>(v);
  const int o = ((j - k) << 3) + k;
  const int ob = o + (o >> 3);
#pragma unroll
  for (int q = 0; q < 8; ++q) out[ob + q * WS] = v[q];
}

// Last pass (radix 8, 4 or 2) from `in` into the registers x.
template <typename T, int SIGN, int L, bool TWC>
__device__ __forceinline__ void gpass_last(cplx<T> (&x)[8], const cplx<T>* in, int j,
                                           const cplx<T>* __restrict__ tw) {
  constexpr int G = 1 << (L - 3), NP = (L + 2) / 3, P = NP - 1;
  constexpr int LNS = 3 * P, NS = 1 << LNS, LR = L - LNS, R = 1 << LR, NB = 8 / R;
  constexpr int RS = (G * NB) + (G * NB) / 8;  // distance of N/R positions (a multiple of 8)
  cplx<T> v[8];
#pragma unroll
  for (int u = 0; u < NB; ++u) {
    const int jj = u * G + j;
    const int k = jj & (NS - 1);
    const int rb = jj + (jj >> 3);
#pragma unroll
    for (int r = 0; r < R; ++r) v[u * R + r] = in[rb + r * RS];
    cplx<T> wr[8];
    twiddles_ct<T, SIGN, R, LNS, TWC>(wr, k, tw);
#pragma unroll
    for (int r = 1; r < R; ++r) v[u * R + r] = cmul<T>(v[u * R + r], wr[r]);
  }
#pragma unroll
  for (int u = 0; u < NB; ++u) {
    dft_r<T, SIGN, R>(v + u * R);
#pragma unroll
    for (int q = 0; q < R; ++q) x[u + q * NB] = v[u * R + q];
  }
}

template <typename T, int SIGN, int L, int P, int SYNC, bool TWC>
__device__ __forceinline__ void gpass_mid(cplx<T>* buf0, cplx<T>* buf1, int& w, int j, int grp,
                                          const cplx<T>* __restrict__ tw) {
  constexpr int NP = (L + 2) / 3;
  if constexpr (P < NP - 1) {
    gpass8<T, SIGN, L, P, TWC>(w ? buf1 : buf0, w ? buf0 : buf1, j, tw);
    gsync<SYNC, (1 << (L - 3))>(grp);
    w ^= 1;
    gpass_mid<T, SIGN, L, P + 1, SYNC, TWC>(buf0, buf1, w, j, grp, tw);
  }
}

// The transform of x (positions j + m G in, positions j + m G out); w selects
// the exchange buffer that is free to write and is left pointing at the
// buffer not read last.
template <typename T, int SIGN, int L, int SYNC, bool TWC>
__device__ __forceinline__ void gfft(cplx<T> (&x)[8], cplx<T>* buf0, cplx<T>* buf1, int& w, int j, int grp,
                                     const cplx<T>* __restrict__ tw) {
  static_assert(L >= 4 && L <= 11, "transform length 16..2048");
  constexpr int G = 1 << (L - 3);
  dft8<T, SIGN>(x);
  {
    cplx<T>* out = w ? buf1 : buf0;
    const int b = 9 * j;  // sidx(8 j + q) = 9 j + q
#pragma unroll
    for (int q = 0; q < 8; ++q) out[b + q] = x[q];
  }
  gsync<SYNC, G>(grp);
  gpass_mid<T, SIGN, L, 1, SYNC, TWC>(buf0, buf1, w, j, grp, tw);
  gpass_last<T, SIGN, L, TWC>(x, w ? buf1 : buf0, j, tw);
  w ^= 1;
}

// Host: the pass-ordered twiddle table of an N-point transform (N - 1
// entries, FP64).
inline void fft_twiddle_table(int log2N, double* re, double* im) {
  const double twopi = 6.283185307179586476925286766559;
  int lNs = 0;
  for (int p = 0; p < fft_num_passes(log2N); ++p) {
    const int lr = fft_pass_lr(log2N, p);
    const int Ns = 1 << lNs, R = 1 << lr;
    for (int r = 1; r < R; ++r)
      for (int k = 0; k < Ns; ++k) {
        const double a = twopi * (double)(r * k) / (double)(Ns * R);
        re[r * Ns + k - 1] = std::cos(a);
        im[r * Ns + k - 1] = -std::sin(a);
      }
    lNs += lr;
  }
}

}  // namespace lm
