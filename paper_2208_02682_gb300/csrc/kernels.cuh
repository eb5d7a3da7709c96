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
// Column pass, inverse: out[o] = IFFT_y( op(src) ) for a tile of 4 kx columns.
// grid (KXP/4, nout), block 4*N/8 threads, smem 4*pad8(N) complex.
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
  cplx<T>* buf = reinterpret_cast<cplx<T>*>(smem_raw);
  const Geom& g = a.g;
  const int N = g.N, K = g.K, KXP = g.KXP;
  const int bst = pad8(N);
  const int o = blockIdx.y;
  const int kx0 = blockIdx.x * 4;
  const int nthr = blockDim.x, tid = threadIdx.x;
  for (int i = tid; i < 4 * bst; i += nthr) buf[i] = mk<T>(0, 0);
  __syncthreads();
  const cplx<T>* s1 = a.src + (long long)a.src_idx[o] * g.ms;
  const cplx<T>* s2 = a.src + (long long)(a.src2_idx[o] < 0 ? a.src_idx[o] : a.src2_idx[o]) * g.ms;
  const int op = a.op[o];
  for (int e = tid; e < g.NY * 4; e += nthr) {
    const int kyi = e >> 2, c = e & 3;
    const int kx = kx0 + c;
    const int ky = kyi - K;
    const long long m = (long long)kyi * KXP + kx;
    cplx<T> v = mk<T>(0, 0);
    if (kx <= K) {
      cplx<T> x = s1[m];
      if (op == OP_ID) v = x;
      else if (op == OP_DX) v = cik<T>(x, (T)kx);
      else if (op == OP_DY) v = cik<T>(x, (T)ky);
      else {  // curl: i kx v - i ky u, src = u, src2 = v
        cplx<T> y = s2[m];
        v = csub<T>(cik<T>(y, (T)kx), cik<T>(x, (T)ky));
      }
    }
    buf[c * bst + pad8(ky & (N - 1))] = v;
  }
  __syncthreads();
  block_fft<T, +1>(buf, g.log2N, bst, a.tw);
  cplx<T>* d = a.dst + (long long)a.dst_idx[o] * g.mi;
  for (int e = tid; e < N * 4; e += nthr) {
    const int n = e >> 2, c = e & 3;
    d[(long long)n * KXP + kx0 + c] = buf[c * bst + pad8(n)];
  }
}

// ---------------------------------------------------------------------------
// Column pass, forward: spectral[o] = FFT_y(mixed[o]) / N, rows |ky| <= K.
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
  cplx<T>* buf = reinterpret_cast<cplx<T>*>(smem_raw);
  const Geom& g = a.g;
  const int N = g.N, K = g.K, KXP = g.KXP;
  const int bst = pad8(N);
  const int o = blockIdx.y;
  const int kx0 = blockIdx.x * 4;
  const int nthr = blockDim.x, tid = threadIdx.x;
  const cplx<T>* s = a.src + (long long)a.src_idx[o] * g.mi;
  for (int e = tid; e < N * 4; e += nthr) {
    const int n = e >> 2, c = e & 3;
    buf[c * bst + pad8(n)] = s[(long long)n * KXP + kx0 + c];
  }
  __syncthreads();
  block_fft<T, -1>(buf, g.log2N, bst, a.tw);
  const T inv = (T)1 / (T)N;
  cplx<T>* d = a.dst + (long long)a.dst_idx[o] * g.ms;
  for (int e = tid; e < g.NY * 4; e += nthr) {
    const int kyi = e >> 2, c = e & 3;
    const int kx = kx0 + c;
    const int ky = kyi - K;
    cplx<T> v = mk<T>(0, 0);
    if (kx <= K) v = cscale<T>(buf[c * bst + pad8(ky & (N - 1))], inv);
    d[(long long)kyi * KXP + kx] = v;
  }
}

// ---------------------------------------------------------------------------
// Row helpers.  A block owns B consecutive rows; its FFT buffer holds B
// transforms of length N at stride pad8(N).

// Fill buf with the Hermitian-paired spectrum Z = A + iB of two real rows
// whose kx >= 0 halves are mixed fields a and b (b < 0: zero), then inverse
// FFT: afterwards buf[row][x] = a(x) + i b(x).  The kx = 0 imaginary parts
// are dropped, as a real inverse transform does.
template <typename T>
__device__ void row_pair_inverse(cplx<T>* buf, const cplx<T>* __restrict__ ma,
                                 const cplx<T>* __restrict__ mb, int row0, int B,
                                 const Geom& g, const cplx<T>* __restrict__ tw) {
  const int N = g.N, K = g.K, KXP = g.KXP;
  const int bst = pad8(N);
  const int nthr = blockDim.x, tid = threadIdx.x;
  for (int i = tid; i < B * bst; i += nthr) buf[i] = mk<T>(0, 0);
  __syncthreads();
  for (int e = tid; e < B * (K + 1); e += nthr) {
    const int r = e / (K + 1), k = e - r * (K + 1);
    const long long off = (long long)(row0 + r) * KXP + k;
    cplx<T> A = ma[off];
    cplx<T> Bv = mb ? mb[off] : mk<T>(0, 0);
    cplx<T>* z = buf + r * bst;
    if (k == 0) {
      z[0] = mk<T>(A.x, Bv.x);
    } else {
      // Z(k) = A + iB, Z(N-k) = conj(A) + i conj(B)
      z[pad8(k)] = mk<T>(A.x - Bv.y, A.y + Bv.x);
      z[pad8(N - k)] = mk<T>(A.x + Bv.y, -A.y + Bv.x);
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
  const int bst = pad8(N);
  const int nthr = blockDim.x, tid = threadIdx.x;
  __syncthreads();
  block_fft<T, -1>(buf, g.log2N, bst, tw);
  const T h = (T)0.5 / (T)N;
  for (int e = tid; e < B * KXP; e += nthr) {
    const int r = e / KXP, k = e - r * KXP;
    const cplx<T>* z = buf + r * bst;
    cplx<T> P = mk<T>(0, 0), Q = mk<T>(0, 0);
    if (k <= K) {
      cplx<T> z1 = z[pad8(k)];
      cplx<T> z2 = z[pad8((N - k) & (N - 1))];
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

// ---------------------------------------------------------------------------
// Row pass, inverse: physical outputs from pairs of mixed fields, with an
// affine epilogue out = scale*val + ax*x + ay*y (used for the mean positions).
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
      const cplx<T> v = buf[r * (pad8(N)) + pad8(x)];
      const long long off = (long long)y * N + x;
      if (a.oa[p] >= 0)
        a.dst[a.oa[p] * a.dst_stride + off] =
            (TO)(a.sa[p] * (double)v.x + a.axa[p] * (x * dxg) + a.aya[p] * (y * dxg));
      if (a.ob[p] >= 0)
        a.dst[a.ob[p] * a.dst_stride + off] =
            (TO)(a.sb[p] * (double)v.y + a.axb[p] * (x * dxg) + a.ayb[p] * (y * dxg));
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
      buf[r * pad8(N) + pad8(x)] = mk<T>((T)pa[off], pb ? (T)pb[off] : (T)0);
    }
    row_pair_forward_store<T>(buf, a.dst + (long long)a.oa[p] * g.mi,
                              a.ob[p] >= 0 ? a.dst + (long long)a.ob[p] * g.mi : nullptr,
                              row0, B, g, a.tw);
  }
}

// ---------------------------------------------------------------------------
// Interval time of a stage: s = (steps done + c_stage) * dt, from the device
// step counter (never accumulated).
__device__ __forceinline__ double stage_time(const long long* ctr, int stage, double dt) {
  const double c = stage == 0 ? 0.0 : (stage == 3 ? 1.0 : 0.5);
  return ((double)(*ctr) + c) * dt;
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
  const T f00 = f[j0 * N + i0], f01 = f[j0 * N + i1];
  const T f10 = f[j1 * N + i0], f11 = f[j1 * N + i1];
  return ((T)1 - ax) * ((T)1 - ay) * f00 + ax * ((T)1 - ay) * f01 +
         ((T)1 - ax) * ay * f10 + ax * ay * f11;
}

// ---------------------------------------------------------------------------
// Row pass with products.  grid (N/B, ceil(npairs/ppb)): block (x, y) owns B
// rows and product pairs [y*ppb, (y+1)*ppb).  Smem: W, P (B*pad8(N) complex
// each), U (4*B*N reals: u, v, h, zeta), XI (2*B*N reals, Strategy 2).
template <typename T>
struct RowProdArgs {
  const cplx<T>* mix;   // column-pass outputs, stride mi
  cplx<T>* prod;        // product mixed fields, stride mi
  const T* phys;        // Strategy 2: physical u, v, h, zeta, q (stride np)
  const long long* ctr; // device step counter
  const cplx<T>* tw;
  Geom g;
  Layout L;
  StepConsts c;
  int B;    // rows per block
  int ppb;  // product pairs per block
  int stage;
};

template <typename T>
__global__ void __launch_bounds__(256) k_row_prod(const __grid_constant__ RowProdArgs<T> a) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const Geom& g = a.g;
  const Layout& L = a.L;
  const int N = g.N, B = a.B;
  const int bst = pad8(N);
  cplx<T>* W = reinterpret_cast<cplx<T>*>(smem_raw);
  cplx<T>* P = W + B * bst;
  T* U = reinterpret_cast<T*>(P + B * bst);
  T* XI = U + 4 * B * N;
  const int row0 = blockIdx.x * B;
  const int p0 = blockIdx.y * a.ppb * 2;
  const int p1 = min(L.np, p0 + a.ppb * 2);
  const int nthr = blockDim.x, tid = threadIdx.x;
  const int BN = B * N;
  const bool kin = L.model == 1;
  const T adv_x = (T)a.c.adv_x, adv_y = (T)a.c.adv_y;
  const T f0 = (T)a.c.f0;
  const double s = stage_time(a.ctr, a.stage, a.c.dt);
  const bool s0 = !(s > 0.0);
  const T inv_s = s0 ? (T)0 : (T)(1.0 / s);
  const T inv_dx = (T)((double)N / 6.283185307179586476925286766559);

  // which physical base fields this block's products read
  bool need_uv = false, need_hz = false;
  for (int p = p0; p < p1; ++p) {
    const int k = L.pk[p];
    if (k == PK_ZV || k == PK_ZU || k == PK_HU || k == PK_HV || k == PK_Q) need_hz = true;
    if (k == PK_ZV || k == PK_ZU || k == PK_KE || k == PK_HU || k == PK_HV) need_uv = true;
    if ((k == PK_ADV || k == PK_XI || k == PK_GBAR) && !kin) need_uv = true;
  }
  // phase 0: physical u, v, h, zeta of the block's rows
  if (L.strategy == 2) {
    for (int e = tid; e < BN; e += nthr) {
      const long long off = (long long)row0 * N + e;
#pragma unroll
      for (int f = 0; f < 4; ++f) U[f * BN + e] = a.phys[f * g.np + off];
    }
    row_pair_inverse<T>(W, a.mix + (long long)L.i_xi[0] * g.mi, a.mix + (long long)L.i_xi[1] * g.mi,
                        row0, B, g, a.tw);
    for (int e = tid; e < BN; e += nthr) {
      const int r = e >> g.log2N, x = e & (N - 1);
      const cplx<T> v = W[r * bst + pad8(x)];
      XI[e] = v.x;
      XI[BN + e] = v.y;
    }
  } else {
    if (need_uv) {
      row_pair_inverse<T>(W, a.mix + (long long)L.i_u * g.mi, a.mix + (long long)L.i_v * g.mi, row0, B, g,
                          a.tw);
      for (int e = tid; e < BN; e += nthr) {
        const int r = e >> g.log2N, x = e & (N - 1);
        const cplx<T> v = W[r * bst + pad8(x)];
        U[e] = v.x;
        U[BN + e] = v.y;
      }
      __syncthreads();
    }
    if (need_hz) {
      row_pair_inverse<T>(W, a.mix + (long long)L.i_h * g.mi, a.mix + (long long)L.i_z * g.mi, row0, B, g,
                          a.tw);
      for (int e = tid; e < BN; e += nthr) {
        const int r = e >> g.log2N, x = e & (N - 1);
        const cplx<T> v = W[r * bst + pad8(x)];
        U[2 * BN + e] = v.x;
        U[3 * BN + e] = v.y;
      }
    }
  }
  __syncthreads();

  // products, two at a time through the forward FFT
  int slot = 0;
  int pend = -1;
  for (int p = p0; p < p1; ++p) {
    const int kind = L.pk[p];
    const bool need_grad = kind == PK_ADV || kind == PK_XI || kind == PK_GBAR;
    if (need_grad) {
      row_pair_inverse<T>(W, a.mix + (long long)L.pa[p] * g.mi, a.mix + (long long)L.pb[p] * g.mi, row0, B,
                          g, a.tw);
    }
    for (int e = tid; e < BN; e += nthr) {
      const int r = e >> g.log2N, x = e & (N - 1);
      const T u = U[e], v = U[BN + e], h = U[2 * BN + e], z = U[3 * BN + e];
      T val;
      switch (kind) {
        case PK_ZV: val = z * v; break;
        case PK_ZU: val = z * u; break;
        case PK_KE: val = (T)0.5 * (u * u + v * v); break;
        case PK_HU: val = h * u; break;
        case PK_HV: val = h * v; break;
        case PK_Q: val = (f0 + z) / h; break;
        case PK_ADV: {
          const cplx<T> d = W[r * bst + pad8(x)];
          const T ua = kin ? adv_x : u, va = kin ? adv_y : v;
          val = ua * d.x + va * d.y;
          break;
        }
        default: {  // PK_XI, PK_GBAR (Strategy 2)
          const cplx<T> d = W[r * bst + pad8(x)];
          const T xx = XI[e], xy = XI[BN + e];
          const T ua = kin ? adv_x : u, va = kin ? adv_y : v;
          const T wx = s0 ? (T)0.5 * ua : xx * inv_s;
          const T wy = s0 ? (T)0.5 * va : xy * inv_s;
          const T wg = wx * d.x + wy * d.y;
          const int c = L.pc[p];
          const int y = row0 + r;
          if (kind == PK_XI) {
            T ui;
            if (kin) ui = c == 0 ? adv_x : adv_y;
            else ui = bilinear<T>(a.phys + (long long)c * g.np, x, y, xx, xy, inv_dx, N);
            val = ui - (c == 0 ? wx : wy) - wg;
          } else {
            const T fi = bilinear<T>(a.phys + (long long)c * g.np, x, y, xx, xy, inv_dx, N);
            val = fi - wg;
          }
          break;
        }
      }
      cplx<T>& dstv = P[r * bst + pad8(x)];
      if (slot == 0) dstv = mk<T>(val, (T)0);
      else dstv.y = val;
    }
    if (slot == 0) {
      pend = p;
      slot = 1;
    } else {
      row_pair_forward_store<T>(P, a.prod + (long long)pend * g.mi, a.prod + (long long)p * g.mi, row0, B,
                                g, a.tw);
      slot = 0;
    }
    __syncthreads();
  }
  if (slot == 1) row_pair_forward_store<T>(P, a.prod + (long long)pend * g.mi, nullptr, row0, B, g, a.tw);
}

// q = (f0 + zeta)/h into the Strategy-2 gather buffer.
template <typename T>
__global__ void k_phys_q(T* phys, long long np, double f0) {
  const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < np) phys[PH_Q * np + i] = ((T)f0 + phys[PH_Z * np + i]) / phys[PH_H * np + i];
}

// ---------------------------------------------------------------------------
// Right-hand sides and RK4 with integrating factor, per spectral mode.
//   stage 0: a = N(y_n)      acc = E^2 a            y1 = E (y_n + dt/2 a)
//   stage 1: b = N(y1)       acc += 2 E b           y2 = E y_n + dt/2 b
//   stage 2: c = N(y2)       acc += 2 E c           y3 = E^2 y_n + dt E c
//   stage 3: d = N(y3)       y_{n+1} = E^2 y_n + dt/6 (acc + d)
// with E = exp(-nu |k|^8 dt/2).  Stage inputs alternate between two buffers:
// a thread reads other fields' stage inputs at its mode, so the next stage's
// values go to the other buffer.
template <typename T>
struct UpdateArgs {
  cplx<T>* y;           // state at t_n
  const cplx<T>* ysin;  // stage input (stage 0: unused, y is the input)
  cplx<T>* ys;          // next stage input (stages 0-2); never aliases ysin
  cplx<T>* acc;
  cplx<T>* comp;  // Kahan compensation (FP32 mode), may be null
  const cplx<T>* ps;  // spectral products
  const T* ef;        // E tables: [IF_DYN][ms], [IF_LM][ms]
  long long* ctr;
  unsigned int* ticket;
  Geom g;
  Layout L;
  StepConsts c;
  int stage;
};

template <typename T>
__device__ __forceinline__ T kahan_add(T sum, T add, T& comp) {
  // compensated sum: returns sum + add, comp carries the lost low part
  const T yk = add - comp;
  const T t = sum + yk;
  comp = (t - sum) - yk;
  return t;
}
__device__ __forceinline__ float kahan_add_rn(float sum, float add, float& comp) {
  const float yk = __fsub_rn(add, comp);
  const float t = __fadd_rn(sum, yk);
  comp = __fsub_rn(__fsub_rn(t, sum), yk);
  return t;
}
__device__ __forceinline__ double kahan_add_rn(double sum, double add, double& comp) {
  const double yk = __dsub_rn(add, comp);
  const double t = __dadd_rn(sum, yk);
  comp = __dsub_rn(__dsub_rn(t, sum), yk);
  return t;
}

// One thread per (mode, evolved field): grid (ceil(ms/256), nf).
template <typename T>
__global__ void __launch_bounds__(256) k_update(const __grid_constant__ UpdateArgs<T> a) {
  const Geom& g = a.g;
  const Layout& L = a.L;
  const long long m = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  const int f = blockIdx.y;
  const double sd = stage_time(a.ctr, a.stage, a.c.dt);
  if (m < g.ms) {
    const int kyi = (int)(m / g.KXP), kx = (int)(m - (long long)kyi * g.KXP);
    if (kx <= g.K) {
      const T kxf = (T)kx, kyf = (T)(kyi - g.K);
      const T dt = (T)a.c.dt;
      const cplx<T>* yin = a.stage == 0 ? a.y : a.ysin;
      const int role = L.frole[f], slot = L.fslot[f];
      cplx<T> r;
      if (role <= R_H) {
        // shallow-water right-hand side, Eq. (sw_eqs_dimless)
        if (L.model == 0) {
          if (role == R_H) {
            r = csub<T>(mk<T>(0, 0), cadd<T>(cik<T>(a.ps[L.p_hu * g.ms + m], kxf), cik<T>(a.ps[L.p_hv * g.ms + m], kyf)));
          } else {
            const cplx<T> hh = yin[L.f_h * g.ms + m];
            const cplx<T> B = cadd<T>(cscale<T>(hh, (T)a.c.c2), a.ps[L.p_ke * g.ms + m]);
            if (role == R_U)
              r = csub<T>(cadd<T>(cscale<T>(yin[L.f_v * g.ms + m], (T)a.c.f0), a.ps[L.p_zv * g.ms + m]), cik<T>(B, kxf));
            else
              r = csub<T>(csub<T>(cscale<T>(yin[L.f_u * g.ms + m], -(T)a.c.f0), a.ps[L.p_zu * g.ms + m]), cik<T>(B, kyf));
          }
        } else {
          const T kc = kxf * (T)a.c.adv_x + kyf * (T)a.c.adv_y;
          r = cik<T>(yin[f * g.ms + m], -kc);
        }
      } else if (role == R_P) {
        const cplx<T> pp = a.ps[L.p_p[slot] * g.ms + m];
        if (L.strategy == 1) {
          // d_t D = s u - u.grad D
          const T s = (T)sd;
          cplx<T> ua;
          if (L.model == 1) {
            const bool k0 = (kx == 0 && kyi == g.K);
            ua = mk<T>(k0 ? (T)(slot == 0 ? a.c.adv_x : a.c.adv_y) : (T)0, 0);
          } else {
            ua = yin[(slot == 0 ? L.f_u : L.f_v) * g.ms + m];
          }
          r = csub<T>(cscale<T>(ua, s), pp);
        } else {
          r = pp;  // xi: the product already holds u(x+xi) - w - w.grad xi
        }
      } else {
        // f_hat of the averaged scalar at this stage
        const int sc = L.lmf[slot];
        cplx<T> fh;
        if (sc == LMF_ZETA) fh = csub<T>(cik<T>(yin[L.f_v * g.ms + m], kxf), cik<T>(yin[L.f_u * g.ms + m], kyf));
        else if (sc == LMF_H) fh = yin[L.f_h * g.ms + m];
        else if (sc == LMF_U) fh = yin[L.f_u * g.ms + m];
        else if (sc == LMF_V) fh = yin[L.f_v * g.ms + m];
        else fh = a.ps[L.p_q * g.ms + m];
        if (role == R_E) {
          r = fh;  // Eq. (ave)
        } else {
          const cplx<T> pg = a.ps[L.p_g[slot] * g.ms + m];
          // S1: f - u.grad g (Eq. gtilde-evol); S2: f(x+xi) - w.grad g
          r = L.strategy == 1 ? csub<T>(fh, pg) : pg;
        }
      }
      // RK4 with integrating factor
      const int cls = L.fclass[f];
      const T E = cls == IF_NONE ? (T)1 : a.ef[cls * g.ms + m];
      const long long o = f * g.ms + m;
      const cplx<T> yn = a.y[o];
      if (a.stage == 0) {
        a.acc[o] = cscale<T>(r, E * E);
        a.ys[o] = cscale<T>(cadd<T>(yn, cscale<T>(r, (T)0.5 * dt)), E);
      } else if (a.stage == 1) {
        a.acc[o] = cadd<T>(a.acc[o], cscale<T>(r, (T)2 * E));
        a.ys[o] = cadd<T>(cscale<T>(yn, E), cscale<T>(r, (T)0.5 * dt));
      } else if (a.stage == 2) {
        a.acc[o] = cadd<T>(a.acc[o], cscale<T>(r, (T)2 * E));
        a.ys[o] = cadd<T>(cscale<T>(yn, E * E), cscale<T>(r, dt * E));
      } else {
        const cplx<T> inc = cscale<T>(cadd<T>(a.acc[o], r), dt / (T)6);
        const T E2 = E * E;
        if (a.comp && L.fkahan[f]) {
          cplx<T> cc = a.comp[o];
          cc.x *= E2;
          cc.y *= E2;
          cplx<T> out;
          out.x = kahan_add_rn(yn.x * E2, inc.x, cc.x);
          out.y = kahan_add_rn(yn.y * E2, inc.y, cc.y);
          a.y[o] = out;
          a.comp[o] = cc;
        } else {
          a.y[o] = cadd<T>(cscale<T>(yn, E2), inc);
        }
      }
    }
  }
  if (a.stage == 3) {
    // the last block to finish advances the step counter (every block has
    // read it above, before taking its ticket)
    __syncthreads();
    if (threadIdx.x == 0) {
      __threadfence();
      const unsigned t = atomicAdd(a.ticket, 1u);
      if (t == gridDim.x * gridDim.y - 1) {
        *a.ticket = 0u;
        *a.ctr = *a.ctr + 1;
        __threadfence();
      }
    }
  }
}

// ---------------------------------------------------------------------------
// Spectral FP64 copy of selected fields, value = (y - comp) * scale.
template <typename T>
__global__ void k_spec_to_f64(const cplx<T>* __restrict__ y, const cplx<T>* __restrict__ comp,
                              double2* __restrict__ out, long long ms, int nsel, const int* sel_unused,
                              int f0_idx, int f1_idx, double scale) {
  (void)sel_unused;
  (void)nsel;
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
