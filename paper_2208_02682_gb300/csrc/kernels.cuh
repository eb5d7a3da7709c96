// kernels.cuh -- GB300 kernels of one RK stage and of the transforms around it.
//
// One RK4 stage of the coupled shallow-water + Lagrangian-mean system is
//   col_inv   spectral state -> mixed fields   (derivatives, inverse y-FFT)
//   row_prod  mixed fields -> products          (inverse x-FFT, physical-space
//             products of the shallow-water equations and of the
//             Lagrangian-mean PDEs, forward x-FFT)
//   col_fwd   products -> spectral products     (forward y-FFT, 2/3 mask)
//   update    right-hand sides and the RK4 integrating-factor combination
// (Strategy 2 adds row_inv into a physical gather buffer before row_prod.)
// The dealiased pseudospectral method is the one the paper uses for both the
// dynamics and the mean equations (Sec. 4.1, 4.2).
#pragma once
#include "common.cuh"
#include "fft.cuh"

namespace lm {

// ---------------------------------------------------------------------------
// Column passes on a tile of C = 2^lC consecutive kx columns (kx0 a multiple
// of C, KXP a multiple of C), C*N/8 threads, smem C*col_stride(N, C) complex.  The
// tile's global accesses are C-wide contiguous runs along kx.

// inverse: d = IFFT_y(op(s1[, s2])), op in {id, d_x, d_y, curl}, zero-padded
// outside |ky| <= K.
template <typename T>
__device__ void col_inverse_tile(cplx<T>* buf, const cplx<T>* __restrict__ s1, const cplx<T>* __restrict__ s2,
                                 int op, cplx<T>* __restrict__ d, const Geom& g, int lC, int kx0,
                                 const cplx<T>* __restrict__ tw) {
  const int N = g.N, K = g.K, KXP = g.KXP;
  const int C = 1 << lC, bst = col_stride<T>(N, C);
  const int nthr = blockDim.x, tid = threadIdx.x;
  // every element written once: op(S) at n = ky mod N for |ky| <= K, else 0
  for (int e = tid; e < N * C; e += nthr) {
    const int n = e >> lC, c = e & (C - 1);
    const int kx = kx0 + c;
    const int ky = n <= K ? n : n - N;
    cplx<T> v = mk<T>(0, 0);
    if (kx <= K && (n <= K || n >= N - K)) {
      const long long m = (long long)(ky + K) * KXP + kx;
      cplx<T> x = s1[m];
      if (op == OP_ID) v = x;
      else if (op == OP_DX) v = cik<T>(x, (T)kx);
      else if (op == OP_DY) v = cik<T>(x, (T)ky);
      else {  // curl: i kx v - i ky u, s1 = u, s2 = v
        cplx<T> y = s2[m];
        v = csub<T>(cik<T>(y, (T)kx), cik<T>(x, (T)ky));
      }
    }
    buf[c * bst + sidx<T>(n)] = v;
  }
  __syncthreads();
  block_fft<T, +1, true>(buf, g.log2N, bst, tw);
  for (int e = tid; e < N * C; e += nthr) {
    const int n = e >> lC, c = e & (C - 1);
    d[(long long)n * KXP + kx0 + c] = buf[c * bst + sidx<T>(n)];
  }
}

// forward: d = FFT_y(s)/N on the rows |ky| <= K (zero for kx > K).
template <typename T>
__device__ void col_forward_tile(cplx<T>* buf, const cplx<T>* __restrict__ s, cplx<T>* __restrict__ d,
                                 const Geom& g, int lC, int kx0, const cplx<T>* __restrict__ tw) {
  const int N = g.N, K = g.K, KXP = g.KXP;
  const int C = 1 << lC, bst = col_stride<T>(N, C);
  const int nthr = blockDim.x, tid = threadIdx.x;
  for (int e = tid; e < N * C; e += nthr) {
    const int n = e >> lC, c = e & (C - 1);
    buf[c * bst + sidx<T>(n)] = s[(long long)n * KXP + kx0 + c];
  }
  __syncthreads();
  block_fft<T, -1, true>(buf, g.log2N, bst, tw);
  const T inv = (T)1 / (T)N;
  for (int e = tid; e < g.NY * C; e += nthr) {
    const int kyi = e >> lC, c = e & (C - 1);
    const int kx = kx0 + c;
    const int ky = kyi - K;
    cplx<T> v = mk<T>(0, 0);
    if (kx <= K) v = cscale<T>(buf[c * bst + sidx<T>(ky & (N - 1))], inv);
    d[(long long)kyi * KXP + kx] = v;
  }
}

// Generic column passes over explicit field lists (initial condition, output
// transforms): grid (KXP/4, nout), 4 columns per block.
template <typename T>
struct ColInvArgs {
  const cplx<T>* src;  // spectral fields, stride ms
  cplx<T>* dst;        // mixed fields, stride mi
  const cplx<T>* tw;
  Geom g;
  int nout;
  int src_idx[MAXI], src2_idx[MAXI], op[MAXI], dst_idx[MAXI];
};

template <typename T>
__global__ void __launch_bounds__(1024) k_col_inv(const __grid_constant__ ColInvArgs<T> a) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const int o = blockIdx.y;
  const cplx<T>* s1 = a.src + (long long)a.src_idx[o] * a.g.ms;
  const cplx<T>* s2 = a.src + (long long)(a.src2_idx[o] < 0 ? a.src_idx[o] : a.src2_idx[o]) * a.g.ms;
  col_inverse_tile<T>(reinterpret_cast<cplx<T>*>(smem_raw), s1, s2, a.op[o], a.dst + (long long)a.dst_idx[o] * a.g.mi,
                      a.g, 2, blockIdx.x * 4, a.tw);
}

template <typename T>
struct ColFwdArgs {
  const cplx<T>* src;  // mixed, stride mi
  cplx<T>* dst;        // spectral, stride ms
  const cplx<T>* tw;
  Geom g;
  int nout;
  int src_idx[MAXP + 8], dst_idx[MAXP + 8];
};

template <typename T>
__global__ void __launch_bounds__(1024) k_col_fwd(const __grid_constant__ ColFwdArgs<T> a) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const int o = blockIdx.y;
  col_forward_tile<T>(reinterpret_cast<cplx<T>*>(smem_raw), a.src + (long long)a.src_idx[o] * a.g.mi,
                      a.dst + (long long)a.dst_idx[o] * a.g.ms, a.g, 2, blockIdx.x * 4, a.tw);
}

// ---------------------------------------------------------------------------
// Row helpers.  A block owns B consecutive rows; its FFT buffer holds B
// transforms of length N at stride row_stride(N).

// Fill buf with the Hermitian-paired spectrum Z = A + iB of two real rows
// whose kx >= 0 halves are mixed fields a and b (b < 0: zero), then inverse
// FFT: afterwards buf[row][x] = a(x) + i b(x).  The kx = 0 imaginary parts
// are dropped, as a real inverse transform does.
template <typename T>
__device__ void row_pair_inverse(cplx<T>* buf, const cplx<T>* __restrict__ ma,
                                 const cplx<T>* __restrict__ mb, int row0, int B,
                                 const Geom& g, const cplx<T>* __restrict__ tw) {
  const int N = g.N, K = g.K, KXP = g.KXP;
  const int bst = row_stride<T>(N);
  const int nthr = blockDim.x, tid = threadIdx.x;
  // Z(k) = A + iB and Z(N-k) = conj(A) + i conj(B) for k <= K (each input
  // read once); the band K < n < N-K is zeroed.  The two writes never touch
  // the same element, so no barrier separates them.
  const int nz = N - 2 * K - 1;
  for (int e = tid; e < B * nz; e += nthr) {
    const int r = e / nz, n = K + 1 + (e - r * nz);
    buf[r * bst + sidx<T>(n)] = mk<T>(0, 0);
  }
  for (int e = tid; e < B * (K + 1); e += nthr) {
    const int r = e / (K + 1), k = e - r * (K + 1);
    const long long off = (long long)(row0 + r) * KXP + k;
    const cplx<T> A = ma[off];
    const cplx<T> Bv = mb ? mb[off] : mk<T>(0, 0);
    cplx<T>* z = buf + r * bst;
    if (k == 0) {
      z[0] = mk<T>(A.x, Bv.x);
    } else {
      z[sidx<T>(k)] = mk<T>(A.x - Bv.y, A.y + Bv.x);
      z[sidx<T>(N - k)] = mk<T>(A.x + Bv.y, -A.y + Bv.x);
    }
  }
  __syncthreads();
  block_fft<T, +1>(buf, g.log2N, bst, tw);
}

// Forward FFT of buf (rows holding p(x) + i q(x)) and scatter of the kx in
// [0, KXP) halves of p and q, scaled by 1/N, into mixed fields da and db.
template <typename T>
__device__ void row_pair_forward_store(cplx<T>* buf, cplx<T>* __restrict__ da,
                                       cplx<T>* __restrict__ db, int row0, int B,
                                       const Geom& g, const cplx<T>* __restrict__ tw) {
  const int N = g.N, K = g.K, KXP = g.KXP;
  const int bst = row_stride<T>(N);
  const int nthr = blockDim.x, tid = threadIdx.x;
  __syncthreads();
  block_fft<T, -1>(buf, g.log2N, bst, tw);
  const T h = (T)0.5 / (T)N;
  for (int e = tid; e < B * KXP; e += nthr) {
    const int r = e / KXP, k = e - r * KXP;
    const cplx<T>* z = buf + r * bst;
    cplx<T> P = mk<T>(0, 0), Q = mk<T>(0, 0);
    if (k <= K) {
      cplx<T> z1 = z[sidx<T>(k)];
      cplx<T> z2 = z[sidx<T>((N - k) & (N - 1))];
      // P = (Z(k) + conj Z(N-k))/2, Q = (Z(k) - conj Z(N-k))/(2i)
      P = mk<T>((z1.x + z2.x) * h, (z1.y - z2.y) * h);
      Q = mk<T>((z1.y + z2.y) * h, (z2.x - z1.x) * h);
    }
    const long long off = (long long)(row0 + r) * KXP + k;
    da[off] = P;
    if (db) db[off] = Q;
  }
  __syncthreads();
}

// Group-owned row transforms (one row per group of G = N/8 threads, N = 2^L
// fixed at compile time; thread j holds positions j + m G, see gfft).

// Hermitian-paired spectrum of one row of mixed fields a and b at the
// thread's positions k = j + m G: Z(k) = A(k) + i B(k) for k <= K,
// conj A(N-k) + i conj B(N-k) for k >= N-K, zero in between; the kx = 0
// imaginary parts are dropped, as a real inverse transform does.
template <typename T, int L>
__device__ __forceinline__ void load_pair_spectrum_ct(cplx<T> (&x)[8], const cplx<T>* __restrict__ ma,
                                                      const cplx<T>* __restrict__ mb, long long rowoff, int j,
                                                      int K) {
  constexpr int N = 1 << L, G = N / 8;
  const cplx<T>* ra = ma + rowoff;
  const cplx<T>* rb = mb ? mb + rowoff : nullptr;
#pragma unroll
  for (int m = 0; m < 8; ++m) {
    const int k = j + m * G;
    cplx<T> z = mk<T>(0, 0);
    if (k <= K) {
      const cplx<T> A = ra[k];
      const cplx<T> Bv = rb ? rb[k] : mk<T>(0, 0);
      z = k == 0 ? mk<T>(A.x, Bv.x) : mk<T>(A.x - Bv.y, A.y + Bv.x);
    } else if (k >= N - K) {
      const cplx<T> A = ra[N - k];
      const cplx<T> Bv = rb ? rb[N - k] : mk<T>(0, 0);
      z = mk<T>(A.x + Bv.y, -A.y + Bv.x);
    }
    x[m] = z;
  }
}

// Spectrum Z of p + i q held at the thread's positions -> kx in [0, KXP)
// halves of p and q, scaled by 1/N, into row `rowoff` of mixed fields da and
// db (db null: p only).  One exchange through the free buffer.
template <typename T, int L, int SYNC>
__device__ __forceinline__ void store_pair_spectrum_ct(const cplx<T> (&x)[8], cplx<T>* buf0, cplx<T>* buf1, int& w,
                                                       cplx<T>* __restrict__ da, cplx<T>* __restrict__ db,
                                                       long long rowoff, int j, int grp, int K, int KXP) {
  constexpr int N = 1 << L, G = N / 8;
  cplx<T>* b = w ? buf1 : buf0;
  if constexpr (G % 8 == 0) {
    const int sb = j + (j >> 3);
#pragma unroll
    for (int m = 0; m < 8; ++m) b[sb + m * (G + G / 8)] = x[m];  // sidx(j + m G)
  } else {
#pragma unroll
    for (int m = 0; m < 8; ++m) b[sidx<T>(j + m * G)] = x[m];
  }
  gsync<SYNC, G>(grp);
  const T h = (T)0.5 / (T)N;
  cplx<T>* ra = da + rowoff;
  cplx<T>* rb = db ? db + rowoff : nullptr;
  for (int k = j; k < KXP; k += G) {
    cplx<T> P = mk<T>(0, 0), Q = mk<T>(0, 0);
    if (k <= K) {
      const cplx<T> z1 = b[k + (k >> 3)];
      const int k2 = (N - k) & (N - 1);
      const cplx<T> z2 = b[k2 + (k2 >> 3)];
      // P = (Z(k) + conj Z(N-k))/2, Q = (Z(k) - conj Z(N-k))/(2i)
      P = mk<T>((z1.x + z2.x) * h, (z1.y - z2.y) * h);
      Q = mk<T>((z1.y + z2.y) * h, (z2.x - z1.x) * h);
    }
    ra[k] = P;
    if (rb) rb[k] = Q;
  }
  w ^= 1;
}

// Call f(IntC<L>()) for the run-time length exponent L in [LO, HI]: the
// stage kernels' bodies are compiled once per transform length.
template <int V> struct IntC { static constexpr int value = V; };
template <int LO, int HI, typename F>
__device__ __forceinline__ void dispatch_L(int L, F&& f) {
  if constexpr (LO <= HI) {
    if (L == LO) f(IntC<LO>());
    else dispatch_L<LO + 1, HI>(L, f);
  }
}

// ---------------------------------------------------------------------------
// Row pass, inverse: physical outputs from pairs of mixed fields, with an
// affine epilogue out = scale*val + ax*x + ay*y + c (mean positions; the
// depth h = 1 + eta from the stored perturbation eta).
template <typename T, typename TO>
struct RowInvArgs {
  const cplx<T>* src;  // mixed, stride mi
  TO* dst;             // physical, stride dst_stride
  long long dst_stride;
  const cplx<T>* tw;
  Geom g;
  int B;
  int npairs;
  int a_idx[8], b_idx[8];  // source mixed fields (b: -1 for none)
  int oa[8], ob[8];        // output field indices (-1: skip)
  double sa[8], sb[8];     // scales
  double axa[8], aya[8], axb[8], ayb[8];
  double ca[8], cb[8];  // constant offsets
};

template <typename T, typename TO>
__global__ void __launch_bounds__(256) k_row_inv(const __grid_constant__ RowInvArgs<T, TO> a) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  cplx<T>* buf = reinterpret_cast<cplx<T>*>(smem_raw);
  const Geom& g = a.g;
  const int N = g.N, B = a.B;
  const int row0 = blockIdx.x * B;
  const int nthr = blockDim.x, tid = threadIdx.x;
  const double dxg = 6.283185307179586476925286766559 / (double)N;
  for (int p = 0; p < a.npairs; ++p) {
    const cplx<T>* ma = a.src + (long long)a.a_idx[p] * g.mi;
    const cplx<T>* mb = a.b_idx[p] >= 0 ? a.src + (long long)a.b_idx[p] * g.mi : nullptr;
    row_pair_inverse<T>(buf, ma, mb, row0, B, g, a.tw);
    for (int e = tid; e < B * N; e += nthr) {
      const int r = e / N, x = e - r * N;
      const int y = row0 + r;
      const cplx<T> v = buf[r * row_stride<T>(N) + sidx<T>(x)];
      const long long off = (long long)y * N + x;
      if (a.oa[p] >= 0)
        a.dst[a.oa[p] * a.dst_stride + off] =
            (TO)(a.sa[p] * (double)v.x + a.axa[p] * (x * dxg) + a.aya[p] * (y * dxg) + a.ca[p]);
      if (a.ob[p] >= 0)
        a.dst[a.ob[p] * a.dst_stride + off] =
            (TO)(a.sb[p] * (double)v.y + a.axb[p] * (x * dxg) + a.ayb[p] * (y * dxg) + a.cb[p]);
    }
    __syncthreads();
  }
}

// ---------------------------------------------------------------------------
// Row pass, forward: mixed outputs from pairs of FP64 physical fields.
template <typename T>
struct RowFwdArgs {
  const double* src;  // physical, stride np
  cplx<T>* dst;       // mixed, stride mi
  const cplx<T>* tw;
  Geom g;
  int B;
  int npairs;
  int a_idx[4], b_idx[4], oa[4], ob[4];
};

template <typename T>
__global__ void __launch_bounds__(256) k_row_fwd(const __grid_constant__ RowFwdArgs<T> a) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  cplx<T>* buf = reinterpret_cast<cplx<T>*>(smem_raw);
  const Geom& g = a.g;
  const int N = g.N, B = a.B;
  const int row0 = blockIdx.x * B;
  const int nthr = blockDim.x, tid = threadIdx.x;
  for (int p = 0; p < a.npairs; ++p) {
    const double* pa = a.src + (long long)a.a_idx[p] * g.np;
    const double* pb = a.b_idx[p] >= 0 ? a.src + (long long)a.b_idx[p] * g.np : nullptr;
    for (int e = tid; e < B * N; e += nthr) {
      const int r = e / N, x = e - r * N;
      const long long off = (long long)(row0 + r) * N + x;
      buf[r * row_stride<T>(N) + sidx<T>(x)] = mk<T>((T)pa[off], pb ? (T)pb[off] : (T)0);
    }
    row_pair_forward_store<T>(buf, a.dst + (long long)a.oa[p] * g.mi,
                              a.ob[p] >= 0 ? a.dst + (long long)a.ob[p] * g.mi : nullptr,
                              row0, B, g, a.tw);
  }
}

// ---------------------------------------------------------------------------
// Interval time of a stage: s = (steps done + c_stage) * dt, from the device
// step counter (never accumulated).
// time of a stage in steps: RK4 (0, 1/2, 1/2, 1), Heun (0, 1), Euler (0)
// Computed in the kernel's precision T: sm_103 issues FP64 arithmetic at a
// small fraction of the FP32 rate, so FP32 kernels keep it out of the set-up
// every thread runs.
// The 64-bit step count is converted through its two 31-bit halves (exact
// in FP64 below 2^53 steps, and in FP32 below 2^24).
template <typename T>
__device__ __forceinline__ T stage_time(const long long* ctr, int stage, T dt, int stepper) {
  const long long n = *ctr;
  const T steps = (T)(int)(n >> 31) * (T)2147483648.0 + (T)(int)(n & 0x7fffffffLL);
  const T c = stage == 0 ? (T)0 : (stepper != 0 || stage == 3 ? (T)1 : (T)0.5);
  return (steps + c) * dt;
}

// Bilinear interpolation of the periodic grid field f at (x_i + xi_x, y_j + xi_y)
// (Sec. 4.2.1).  The displacement in cells d = xi/dx gives the cell index
// i + floor(d) and the weight d - floor(d).  Indices wrap with & (N-1), so any
// displacement (even a non-finite one) reads inside the field.
template <typename T>
__device__ __forceinline__ T bilinear(const T* __restrict__ f, int i, int j, T xi_x, T xi_y,
                                      T inv_dx, int N) {
  const T dxc = xi_x * inv_dx, dyc = xi_y * inv_dx;
  const T fx = floor(dxc), fy = floor(dyc);
  const T ax = dxc - fx, ay = dyc - fy;
  const unsigned msk = (unsigned)N - 1u;
  const unsigned i0 = ((unsigned)i + (unsigned)(int)fx) & msk;
  const unsigned j0 = ((unsigned)j + (unsigned)(int)fy) & msk;
  const unsigned i1 = (i0 + 1u) & msk, j1 = (j0 + 1u) & msk;
  const T f00 = __ldg(f + j0 * N + i0), f01 = __ldg(f + j0 * N + i1);
  const T f10 = __ldg(f + j1 * N + i0), f11 = __ldg(f + j1 * N + i1);
  return ((T)1 - ax) * ((T)1 - ay) * f00 + ax * ((T)1 - ay) * f01 +
         ((T)1 - ax) * ay * f10 + ax * ay * f11;
}

// ---------------------------------------------------------------------------
// Two-dimensional Euler model: u, v of the vorticity in slot fh, through the
// streamfunction (u_hat = i ky zeta_hat/|k|^2, v_hat = -i kx zeta_hat/|k|^2,
// zero at k = 0), into slots fu, fv; one thread per box mode.
template <typename T>
__global__ void k_velocity_from_vorticity(cplx<T>* __restrict__ y, Geom g, int fu, int fv, int fh) {
  const long long m = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (m >= g.ms) return;
  const int mi = (int)m;
  const int kyi = mi / g.KXP, kx = mi - kyi * g.KXP;
  const T kxf = (T)kx, kyf = (T)(kyi - g.K);
  const cplx<T> z = y[(long long)fh * g.ms + m];
  const T k2 = kxf * kxf + kyf * kyf;
  const T inv = k2 > (T)0 ? (T)1 / k2 : (T)0;
  y[(long long)fu * g.ms + m] = mk<T>(-kyf * z.y * inv, kyf * z.x * inv);
  y[(long long)fv * g.ms + m] = mk<T>(kxf * z.y * inv, -kxf * z.x * inv);
}

// ---------------------------------------------------------------------------
// Spectral FP64 copy of selected fields, value = (y - comp) * scale.
template <typename T>
__global__ void k_spec_to_f64(const cplx<T>* __restrict__ y, const cplx<T>* __restrict__ comp,
                              double2* __restrict__ out, long long ms, int f0_idx, int f1_idx, double scale) {
  const long long m = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (m >= ms) return;
  const int idx[2] = {f0_idx, f1_idx};
#pragma unroll
  for (int q = 0; q < 2; ++q) {
    if (idx[q] < 0) continue;
    const cplx<T> v = y[idx[q] * ms + m];
    double re = (double)v.x, im = (double)v.y;
    if (comp) {
      const cplx<T> c = comp[idx[q] * ms + m];
      re -= (double)c.x;
      im -= (double)c.y;
    }
    out[q * ms + m] = make_double2(re * scale, im * scale);
  }
}

// Add delta to the real part of one spectral coefficient (mean depth).
__global__ void k_add_real(double2* p, double delta);

// FP64 spectral -> T spectral (initial condition).
template <typename T>
__global__ void k_spec_from_f64(const double2* __restrict__ in, cplx<T>* __restrict__ y, long long n) {
  const long long m = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (m < n) y[m] = mk<T>((T)in[m].x, (T)in[m].y);
}

// ---------------------------------------------------------------------------
// Deterministic FP64 invariant sums over a physical grid (u, v, h, zeta):
// per-block partial sums, then one block adds the partials in fixed order.
__global__ void k_diag_partial(const double* __restrict__ phys, long long np, double f0, double c2,
                               double* __restrict__ part);
__global__ void k_diag_final(const double* __restrict__ part, int nblk, long long np, double* __restrict__ out);

}  // namespace lm
