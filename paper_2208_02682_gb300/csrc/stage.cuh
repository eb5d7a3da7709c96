// stage.cuh -- the kernels of one RK stage, over a batch of independent runs.
//
// Every stage kernel takes a device table of run descriptors and, per kernel
// kind, a prefix sum of the blocks each run needs: block b belongs to the run
// r with start[r] <= b < start[r+1] and works on local block b - start[r].
// A single handle is a batch of one; sw_batch steps many handles (different
// grid sizes, strategies and field sets) in the same launches.  Block shapes
// are uniform within a launch: C*N (columns x points) and Bp*N, Bi*N (rows x
// points) are equal for all members.
//
// Per stage:  col_inv -> [row_inv, phys_q: Strategy 2] -> row_prod -> col_fwd -> update
#pragma once
#include "kernels.cuh"

namespace lm {

enum { KT_COL_INV = 0, KT_ROW_INV = 1, KT_PHYS_Q = 2, KT_ROW_PROD = 3, KT_COL_FWD = 4, KT_UPDATE = 5, KT_COUNT = 6 };

template <typename T>
struct RunDesc {
  Geom g;
  Layout L;
  StepConsts c;
  T cdt, cf0, cc2, cadvx, cadvy;  // dt, f0, c2, adv in the kernels' precision
  cplx<T>* y;     // state at t_n
  cplx<T>* ysa;   // stage inputs of stages 1 and 3
  cplx<T>* ysb;   // stage input of stage 2
  cplx<T>* acc;   // RK accumulator
  cplx<T>* comp;  // Kahan compensation (FP32 mode; null in FP64)
  cplx<T>* ps;    // spectral products
  cplx<T>* mix;   // column-pass outputs (mixed)
  cplx<T>* pmix;  // row-pass products (mixed)
  T* phys;        // Strategy-2 gather buffer
  const T* ef;    // integrating-factor tables
  const cplx<T>* tw;
  long long* ctr;
  unsigned* ticket;
  int lC;         // column tile: C = 2^lC columns
  int Bp, ppb;    // row_prod: rows per block, product pairs per block
  int Wp;         // row_prod: groups of N/8 threads per row
  int Bi;         // row_inv: rows per block
  int nb[KT_COUNT];
};

__device__ __forceinline__ int find_run(const int* __restrict__ start, int nruns, int b) {
  int lo = 0, hi = nruns;
  while (hi - lo > 1) {
    const int mid = (lo + hi) >> 1;
    if (start[mid] <= b) lo = mid;
    else hi = mid;
  }
  return lo;
}

// Copy the block's run descriptor into shared memory with one cooperative
// load, so the kernel's many field-index and pointer lookups are shared-memory
// reads instead of chains of dependent global loads.
template <typename T>
__device__ __forceinline__ const RunDesc<T>& load_desc(const RunDesc<T>* __restrict__ runs, int r,
                                                       unsigned char* sbuf) {
  static_assert(sizeof(RunDesc<T>) % sizeof(int) == 0, "descriptor size");
  const int* src = reinterpret_cast<const int*>(runs + r);
  int* dst = reinterpret_cast<int*>(sbuf);
  constexpr int n = (int)(sizeof(RunDesc<T>) / sizeof(int));
  for (int i = threadIdx.x; i < n; i += blockDim.x) dst[i] = __ldg(src + i);
  __syncthreads();
  return *reinterpret_cast<const RunDesc<T>*>(sbuf);
}

#define LM_STAGE_DESC(T_)                                                 \
  __shared__ __align__(16) unsigned char sdesc_[sizeof(RunDesc<T_>)];   \
  const RunDesc<T_>& d = load_desc<T_>(runs, r, sdesc_)

template <typename T>
__device__ __forceinline__ const cplx<T>* stage_input(const RunDesc<T>& d, int stage) {
  return stage == 0 ? d.y : (stage == 2 ? d.ysb : d.ysa);
}

// ---------------------------------------------------------------------------
// Column passes on group transforms: a block owns a tile of C = 2^lC
// consecutive kx columns; thread t works on column c = t mod C and rows
// n = j + m N/8 (j = t div C, m < 8), so the lanes of a warp read and write
// C-wide contiguous runs of the kx-major fields straight from and to
// registers.  Smem: C * col_buf_stride(N, C) complex.

// Threads per column-pass block at most: C*N/8 is 256 up to 512^2 and in
// FP64; FP32 tiles of 4 columns at 1024^2 and 2048^2 take 512 and 1024.
template <typename T> constexpr int col_max_threads() { return sizeof(T) == 4 ? 1024 : 256; }

// a1: column inverse pass, local block = (output field, kx tile):
// mixed = IFFT_y(op(spectral)) with op in {id, d_x, d_y, curl}, zero-padded
// outside |ky| <= K.
template <typename T>
__global__ void __launch_bounds__(col_max_threads<T>()) k_stage_col_inv(const RunDesc<T>* __restrict__ runs,
                                                       const int* __restrict__ start, int nruns, int stage) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const int r = find_run(start, nruns, blockIdx.x);
  const RunDesc<T>& d = runs[r];
  pdl_wait();  // state written by the previous kernels: only after this
  const int lb = blockIdx.x - start[r];
  dispatch_L<4, 11>(d.g.log2N, [&](auto Lc) {
    constexpr int L = decltype(Lc)::value, N = 1 << L, G = N / 8;
    const int K = d.g.K, KXP = d.g.KXP;
    const int lC = d.lC, C = 1 << lC;
    const int ntile = KXP >> lC;
    const int o = lb / ntile, tile = lb - o * ntile;
    const int c = threadIdx.x & (C - 1), j = threadIdx.x >> lC;
    const int kx = (tile << lC) + c;
    const cplx<T>* src = stage_input(d, stage);
    const int op = d.L.i_op[o];
    const cplx<T>* s1 = src + (long long)d.L.i_src[o] * d.g.ms + kx;
    const cplx<T>* s2 = src + (long long)(d.L.i_src2[o] < 0 ? d.L.i_src[o] : d.L.i_src2[o]) * d.g.ms + kx;
    const bool col = kx <= K;
    cplx<T> x[8];
    int kyv[8];
#pragma unroll
    for (int m = 0; m < 8; ++m) {
      const int n = j + m * G;
      kyv[m] = n <= K ? n : n - N;
      x[m] = mk<T>(0, 0);
      if (col && (n <= K || n >= N - K)) x[m] = s1[(kyv[m] + K) * KXP];
    }
    // the operator is uniform over the block
    if (op == OP_DX) {
#pragma unroll
      for (int m = 0; m < 8; ++m) x[m] = cik<T>(x[m], (T)kx);
    } else if (op == OP_DY) {
#pragma unroll
      for (int m = 0; m < 8; ++m) x[m] = cik<T>(x[m], (T)kyv[m]);
    } else if (op == OP_CURL) {
      // curl: i kx v - i ky u (s1 = u, s2 = v)
#pragma unroll
      for (int m = 0; m < 8; ++m) {
        const int n = j + m * G;
        cplx<T> b = mk<T>(0, 0);
        if (col && (n <= K || n >= N - K)) b = s2[(kyv[m] + K) * KXP];
        x[m] = csub<T>(cik<T>(b, (T)kx), cik<T>(x[m], (T)kyv[m]));
      }
    }
    cplx<T>* b0 = reinterpret_cast<cplx<T>*>(smem_raw) + (size_t)c * col_buf_stride<T>(N, C);
    int w = 0;
    gfft<T, +1, L, 2, false>(x, b0, b0 + row_stride<T>(N), w, j, 0, d.tw);
    cplx<T>* dst = d.mix + (long long)o * d.g.mi + kx;
#pragma unroll
    for (int m = 0; m < 8; ++m) dst[(j + m * G) * KXP] = x[m];
  });
  pdl_release();
}

// a4 (first half): column forward pass of the products, local block =
// (product, kx tile): spectral = FFT_y(mixed)/N on the rows |ky| <= K (zero
// for kx > K).
template <typename T>
__global__ void __launch_bounds__(col_max_threads<T>()) k_stage_col_fwd(const RunDesc<T>* __restrict__ runs,
                                                       const int* __restrict__ start, int nruns) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const int r = find_run(start, nruns, blockIdx.x);
  const RunDesc<T>& d = runs[r];
  pdl_wait();  // state written by the previous kernels: only after this
  const int lb = blockIdx.x - start[r];
  dispatch_L<4, 11>(d.g.log2N, [&](auto Lc) {
    constexpr int L = decltype(Lc)::value, N = 1 << L, G = N / 8;
    const int K = d.g.K, KXP = d.g.KXP;
    const int lC = d.lC, C = 1 << lC;
    const int ntile = KXP >> lC;
    const int p = lb / ntile, tile = lb - p * ntile;
    const int c = threadIdx.x & (C - 1), j = threadIdx.x >> lC;
    const int kx = (tile << lC) + c;
    const cplx<T>* src = d.pmix + (long long)p * d.g.mi + kx;
    cplx<T> x[8];
#pragma unroll
    for (int m = 0; m < 8; ++m) x[m] = src[(j + m * G) * KXP];
    cplx<T>* b0 = reinterpret_cast<cplx<T>*>(smem_raw) + (size_t)c * col_buf_stride<T>(N, C);
    int w = 0;
    gfft<T, -1, L, 2, false>(x, b0, b0 + row_stride<T>(N), w, j, 0, d.tw);
    const T inv = (T)1 / (T)N;
    cplx<T>* dst = d.ps + (long long)p * d.g.ms + kx;
#pragma unroll
    for (int m = 0; m < 8; ++m) {
      const int k = j + m * G;
      if (k <= K || k >= N - K) {
        const int ky = k <= K ? k : k - N;
        dst[(ky + K) * KXP] = kx <= K ? cscale<T>(x[m], inv) : mk<T>(0, 0);
      }
    }
  });
  pdl_release();
}

// ---------------------------------------------------------------------------
// Column forward pass of the large grids (FP32, N = 2^L >= 1024, tiles of
// C = 4 columns: C N/8 = 512 or 1024 threads, two or one blocks per SM).
// With one or two blocks per SM the loads of a tile and the butterflies of
// the previous one cannot overlap across blocks, so this pass is
// persistent: block b takes the launch's work items b, b + gridDim.x, ...
// (an item is the local block of k_stage_col_fwd: (product, tile) of one
// run), and while it transforms one item, the next item's mixed tile is
// copied into shared memory with cp.async (16-byte copies, completed by the
// group wait before the tile is read).  The arithmetic is that of
// k_stage_col_fwd, element for element.  (The same staging for the column
// inverse pass, whose time is set by its 16 output writes rather than its
// reads, measured no faster and is not used.)
// Smem: C exchange-buffer pairs (col_buf_stride), then the staged tile of
// N rows x C complex.
constexpr int PIPE_C = 4;

__device__ __forceinline__ void cp_async16(void* smem, const void* gmem) {
  const unsigned s = static_cast<unsigned>(__cvta_generic_to_shared(smem));
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(s), "l"(gmem) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
__device__ __forceinline__ void cp_async_wait_all() { asm volatile("cp.async.wait_group 0;" ::: "memory"); }

// Copy the mixed tile of work item `item` (N rows x 4 complex, row stride
// KXP) into the staging buffer.
__device__ __forceinline__ void pipe_stage(float2* st, const RunDesc<float>* __restrict__ runs,
                                           const int* __restrict__ start, int nruns, int item) {
  const int r = find_run(start, nruns, item);
  const RunDesc<float>& d = runs[r];
  const int lb = item - start[r];
  const int ntile = d.g.KXP / PIPE_C;
  const int p = lb / ntile, tile = lb - p * ntile;
  const float2* src = d.pmix + (long long)p * d.g.mi + tile * PIPE_C;
  const int rows = d.g.N, KXP = d.g.KXP;
  for (int q = threadIdx.x; q < 2 * rows; q += blockDim.x) {
    const int row = q >> 1, half = q & 1;
    cp_async16(st + row * PIPE_C + half * 2, src + (long long)row * KXP + half * 2);
  }
}

template <int L>
__global__ void __launch_bounds__(1024, 1) k_stage_col_fwd_pipe(const RunDesc<float>* __restrict__ runs,
                                                                const int* __restrict__ start, int nruns,
                                                                int total) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  constexpr int N = 1 << L, G = N / 8, C = PIPE_C;
  float2* xb = reinterpret_cast<float2*>(smem_raw);
  float2* st = xb + (size_t)C * col_buf_stride<float>(N, C);
  const int c = threadIdx.x & (C - 1), j = threadIdx.x >> 2;
  float2* b0 = xb + (size_t)c * col_buf_stride<float>(N, C);
  pdl_wait();  // state written by the previous kernels: only after this
  int item = blockIdx.x;
  if (item < total) pipe_stage(st, runs, start, nruns, item);
  cp_async_commit();
  int w = 0;
  for (; item < total; item += gridDim.x) {
    cp_async_wait_all();
    __syncthreads();  // the staged tile is complete and the last transform's buffers are free
    const int r = find_run(start, nruns, item);
    const RunDesc<float>& d = runs[r];
    const int K = d.g.K, KXP = d.g.KXP;
    const int lb = item - start[r];
    const int ntile = KXP / C;
    const int p = lb / ntile, tile = lb - p * ntile;
    const int kx = tile * C + c;
    float2 x[8];
#pragma unroll
    for (int m = 0; m < 8; ++m) x[m] = st[(j + m * G) * C + c];
    __syncthreads();  // every thread has read the staged tile
    if (item + gridDim.x < total) pipe_stage(st, runs, start, nruns, item + gridDim.x);
    cp_async_commit();
    gfft<float, -1, L, 2, false>(x, b0, b0 + row_stride<float>(N), w, j, 0, d.tw);
    const float inv = 1.0f / (float)N;
    float2* dst = d.ps + (long long)p * d.g.ms + kx;
#pragma unroll
    for (int m = 0; m < 8; ++m) {
      const int k = j + m * G;
      if (k <= K || k >= N - K) {
        const int ky = k <= K ? k : k - N;
        dst[(ky + K) * KXP] = kx <= K ? cscale<float>(x[m], inv) : mk<float>(0, 0);
      }
    }
  }
  cp_async_wait_all();
  pdl_release();
}

// Shared memory of a pipelined column forward launch.
inline size_t col_fwd_pipe_smem(int N) {
  return ((size_t)PIPE_C * col_buf_stride<float>(N, PIPE_C) + (size_t)N * PIPE_C) * sizeof(float2);
}

// a3: Strategy-2 gather buffer (physical u, v | h, zeta), local block =
// (pair, row block of Bi rows, one row per group of N/8 threads).
template <typename T, bool WARP>
__global__ void __launch_bounds__(256) k_stage_row_inv(const RunDesc<T>* __restrict__ runs,
                                                       const int* __restrict__ start, int nruns) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const int r = find_run(start, nruns, blockIdx.x);
  const RunDesc<T>& d = runs[r];
  pdl_wait();  // state written by the previous kernels: only after this
  const int lb = blockIdx.x - start[r];
  auto body = [&](auto Lc) {
    constexpr int L = decltype(Lc)::value, N = 1 << L, G = N / 8;
    constexpr int SYNC = L <= 8 ? 0 : 1;
    const Geom& g = d.g;
    const int B = d.Bi;
    const int nrb = N / B;
    const int pair = lb / nrb, rb = lb - pair * nrb;
    const int grp = threadIdx.x / G, j = threadIdx.x - grp * G;
    const int y = rb * B + grp;
    constexpr int rs = N + N / 8;
    cplx<T>* buf0 = reinterpret_cast<cplx<T>*>(smem_raw) + (size_t)grp * 2 * rs;
    cplx<T>* buf1 = buf0 + rs;
    // pairs (u, v), (h, zeta) and, Strategy 2, (xi_x, xi_y)
    const int ia = pair == 0 ? d.L.i_u : (pair == 1 ? d.L.i_h : d.L.i_xi[0]);
    const int ib = pair == 0 ? d.L.i_v : (pair == 1 ? d.L.i_z : d.L.i_xi[1]);
    const int oa = pair == 0 ? PH_U : (pair == 1 ? PH_H : PH_XX);
    const int ob = pair == 0 ? PH_V : (pair == 1 ? PH_Z : PH_XY);
    cplx<T> x[8];
    int w = 0;
    load_pair_spectrum_ct<T, L>(x, d.mix + (long long)ia * g.mi, d.mix + (long long)ib * g.mi, (long long)y * g.KXP,
                                j, g.K);
    gfft<T, +1, L, SYNC, false>(x, buf0, buf1, w, j, grp, d.tw);
    T* pa = d.phys + (long long)oa * g.np + (long long)y * N + j;
    T* pb = d.phys + (long long)ob * g.np + (long long)y * N + j;
#pragma unroll
    for (int m = 0; m < 8; ++m) {
      pa[m * G] = x[m].x;
      pb[m * G] = x[m].y;
    }
  };
  if constexpr (WARP) dispatch_L<4, 8>(d.g.log2N, body);
  else dispatch_L<4, 11>(d.g.log2N, body);
  pdl_release();
}

// q = (f0 + zeta)/h, h = 1 + eta, into the gather buffer (Strategy 2 with PV
// averaged).
template <typename T>
__global__ void __launch_bounds__(256) k_stage_phys_q(const RunDesc<T>* __restrict__ runs,
                                                      const int* __restrict__ start, int nruns) {
  const int r = find_run(start, nruns, blockIdx.x);
  const RunDesc<T>& d = runs[r];
  pdl_wait();  // state written by the previous kernels: only after this
  const long long i = (long long)(blockIdx.x - start[r]) * blockDim.x + threadIdx.x;
  const long long np = d.g.np;
  if (i < np) d.phys[PH_Q * np + i] = (d.cf0 + d.phys[PH_Z * np + i]) / ((T)1 + d.phys[PH_H * np + i]);
  pdl_release();
}

// ---------------------------------------------------------------------------
// a2: row pass with products.  Local block = (pair group, row block): Bp rows
// and product pairs [pg*ppb, (pg+1)*ppb), with Wp groups of G = N/8 threads
// per row.  Every transform stays in the registers of its group (gfft):
// a row's physical values live at the thread's own positions x = j + m G,
// where the products are formed and the forward transform of each product
// pair starts.  First the row's base fields (u, v, h, zeta; Strategy 2: xi),
// transformed by the row inverse pass, are read into the row's U, the loads
// shared out over the row's groups; then the groups take the block's product
// pairs in turn.  Wp > 1 only when a group is a whole
// number of warps (N >= 256), so groups that do different numbers of
// transforms never share a warp barrier.
// Products are formed in the registers that feed the forward transform of
// their pair: a pair holds at most one product that needs a transform or a
// gather of its own ("heavy", placed first) unless Layout.heavy2 says
// otherwise, so the first product overwrites its gradient pair element by
// element and the second is formed from the base fields beside it.
// Smem: per row U (u, v, h, zeta and, Strategy 2, xi_x, xi_y: N reals each);
// per group two exchange buffers of row_stride(N) complex and
// row_prod_group_rows(L) rows of N reals: Strategy 2, the first product's
// values gathered at x + xi; with heavy2, the first product's values while
// the second is transformed and (Strategy 2) the second product's gathered
// values.

// Threads per row-pass block at most (two blocks per SM: up to 85 registers
// in FP32, 128 in FP64).
template <typename T> constexpr int row_prod_max_threads() { return sizeof(T) == 4 ? 384 : 256; }

__device__ __forceinline__ bool product_heavy(int k) { return k == PK_ADV || k == PK_XI || k == PK_GBAR; }

// Rows of N reals per group of the row pass besides its exchange buffers.
__host__ __device__ __forceinline__ int row_prod_group_rows(const Layout& L) {
  return (L.strategy == 2 ? 1 : 0) + (L.heavy2 ? (L.strategy == 2 ? 2 : 1) : 0);
}

template <typename T, bool WARP>
__global__ void __launch_bounds__(row_prod_max_threads<T>(), 2) k_stage_row_prod(const RunDesc<T>* __restrict__ runs,
                                                                                const int* __restrict__ start,
                                                                                int nruns, int stage) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const int r = find_run(start, nruns, blockIdx.x);
  LM_STAGE_DESC(T);  // field and product lookups from shared memory
  pdl_wait();  // state written by the previous kernels: only after this
  const int lb = blockIdx.x - start[r];
  auto body = [&](auto Lc) {
  constexpr int L_ = decltype(Lc)::value, N = 1 << L_, G = N / 8;
  constexpr int SYNC = L_ <= 8 ? 0 : 1;
  const Geom& g = d.g;
  const Layout& L = d.L;
  const int B = d.Bp, W = d.Wp;
  const int nrb = N / B;
  const int pg = lb / nrb, rb = lb - pg * nrb;
  const int gi = threadIdx.x / G, j = threadIdx.x - gi * G;
  const int row = gi / W, wg = gi - row * W;
  const int y = rb * B + row;
  constexpr int rs = N + N / 8;
  const bool s2 = L.strategy == 2;
  const int nur = s2 ? 6 : 4, nug = row_prod_group_rows(L);
  T* U = reinterpret_cast<T*>(smem_raw) + (size_t)row * nur * N;
  T* XI = U + 4 * N;
  cplx<T>* buf0 = reinterpret_cast<cplx<T>*>(reinterpret_cast<T*>(smem_raw) + (size_t)B * nur * N) +
                  (size_t)gi * (2 * rs + (nug * N) / 2);
  cplx<T>* buf1 = buf0 + rs;
  T* S0 = reinterpret_cast<T*>(buf1 + rs);  // Strategy 2: first product's gathered values
  T* P0 = S0 + (s2 ? N : 0);                // heavy2: first product's values
  T* S1 = P0 + N;                           // heavy2, Strategy 2: second product's gathered values
  const int np = L.np;
  const int p0 = pg * d.ppb * 2;
  const int p1 = min(np, p0 + d.ppb * 2);
  const bool kin = L.model == 1;
  const T adv_x = d.cadvx, adv_y = d.cadvy;
  const T f0 = d.cf0;
  const T s = stage_time<T>(d.ctr, stage, d.cdt, d.c.stepper);
  const bool s0 = !(s > (T)0);
  const T inv_s = s0 ? (T)0 : (T)1 / s;
  // xi-first scheme: gbar steps with the updated xi at its time s + dt
  const bool xf = L.scheme == SCHEME_XI_FIRST;
  const T inv_sg = xf ? (T)1 / (s + d.cdt) : inv_s;
  const T inv_dx = (T)N / (T)6.283185307179586476925286766559;
  const cplx<T>* mix = d.mix;
  // the gather buffer (written by the previous kernel) is read-only here:
  // non-coherent loads that need not wait for this block's shared-memory stores
  const T* __restrict__ phys = d.phys;
  const long long npts = g.np;
  const long long rowoff = (long long)y * g.KXP;
  int w = 0;
  cplx<T> x[8];

  // the row's physical u, v, h, zeta (and, Strategy 2, xi_x, xi_y), written
  // by the row inverse pass, into U (and XI = U + 4N), shared out over the
  // row's groups
  {
    const int nplanes = s2 ? 6 : 4;
#pragma unroll
    for (int f = 0; f < 6; ++f) {
      if (f < nplanes && f % W == wg) {
        const T* __restrict__ src = phys + (long long)(f < 4 ? f : f + 1) * npts + (long long)y * N + j;
        T v[8];
#pragma unroll
        for (int m = 0; m < 8; ++m) v[m] = __ldg(src + m * G);
#pragma unroll
        for (int m = 0; m < 8; ++m) U[f * N + m * G + j] = v[m];
      }
    }
  }

  // the gradient spectrum of a product, into the registers x; the first
  // product of the group's first pair is loaded before the wait for the row's
  // base fields
  const int npair = (p1 - p0 + 1) >> 1;
  auto load_grad = [&](int p) {
    if (product_heavy(L.pk[p]))
      load_pair_spectrum_ct<T, L_>(x, mix + (long long)L.pa[p] * g.mi, mix + (long long)L.pb[p] * g.mi, rowoff, j,
                                   g.K);
  };
  if (wg < npair) load_grad(p0 + 2 * wg);
  __syncthreads();

  // Strategy 2: the values at x + xi (Eqs. xi_evol, barf_xi) that product p
  // needs, by bilinear interpolation into dst (N reals)
  auto gather = [&](int p, T* dst) {
    const int kind = L.pk[p], pc = L.pc[p];
    if (kind != PK_GBAR && (kind != PK_XI || kin)) return;
    const T* __restrict__ src = phys + (long long)pc * npts;
#pragma unroll
    for (int m = 0; m < 8; ++m) {
      const int e = m * G + j;
      dst[e] = bilinear<T>(src, e, y, XI[e], XI[N + e], inv_dx, N);
    }
  };

  // product p at the thread's positions into the real (slot 0) or imaginary
  // (slot 1) parts of x; a heavy product reads its gradient pair from x at
  // the same position first, and (Strategy 2) its gathered values from sv
  auto form = [&](int p, int slot, const T* sv) {
    const int kind = L.pk[p], pc = L.pc[p];
    auto put = [&](int m, T v) {
      if (slot) x[m].y = v;
      else x[m].x = v;
    };
    switch (kind) {
      case PK_ZV:
#pragma unroll
        for (int m = 0; m < 8; ++m) put(m, U[3 * N + m * G + j] * U[N + m * G + j]);
        break;
      case PK_ZU:
#pragma unroll
        for (int m = 0; m < 8; ++m) put(m, U[3 * N + m * G + j] * U[m * G + j]);
        break;
      case PK_KE:
#pragma unroll
        for (int m = 0; m < 8; ++m) {
          const T u = U[m * G + j], v = U[N + m * G + j];
          put(m, (T)0.5 * (u * u + v * v));
        }
        break;
      // depth h = 1 + eta; the state and the row buffers hold eta
      case PK_HU:
#pragma unroll
        for (int m = 0; m < 8; ++m) {
          const T u = U[m * G + j];
          put(m, u + U[2 * N + m * G + j] * u);
        }
        break;
      case PK_HV:
#pragma unroll
        for (int m = 0; m < 8; ++m) {
          const T v = U[N + m * G + j];
          put(m, v + U[2 * N + m * G + j] * v);
        }
        break;
      case PK_Q:
#pragma unroll
        for (int m = 0; m < 8; ++m) put(m, (f0 + U[3 * N + m * G + j]) / ((T)1 + U[2 * N + m * G + j]));
        break;
      case PK_ADV:
        // u.grad G (Eq. gtilde-evol) or u.grad D
#pragma unroll
        for (int m = 0; m < 8; ++m) {
          const T ua = kin ? adv_x : U[m * G + j], va = kin ? adv_y : U[N + m * G + j];
          put(m, ua * x[m].x + va * x[m].y);
        }
        break;
      default: {
        // Strategy 2, Eqs. (xi_evol), (barf_xi): w = xi/s, limit u/2 at s = 0
#pragma unroll
        for (int m = 0; m < 8; ++m) {
          const int e = m * G + j;
          const T xx = XI[e], xy = XI[N + e];
          const T ua = kin ? adv_x : U[e], va = kin ? adv_y : U[N + e];
          const bool sz = s0 && !(xf && kind == PK_GBAR);
          const T is = kind == PK_GBAR ? inv_sg : inv_s;
          const T wx = sz ? (T)0.5 * ua : xx * is;
          const T wy = sz ? (T)0.5 * va : xy * is;
          const T wgrad = wx * x[m].x + wy * x[m].y;
          const T fi = (kind == PK_XI && kin) ? (pc == 0 ? adv_x : adv_y) : sv[e];
          put(m, kind == PK_XI ? fi - (pc == 0 ? wx : wy) - wgrad : fi - wgrad);
        }
        break;
      }
    }
  };

  // product pairs, shared out over the row's groups
  for (int q = wg; q < npair; q += W) {
    const int pa = p0 + 2 * q;
    const int npq = min(2, p1 - pa);
    const bool h2 = npq == 2 && product_heavy(L.pk[pa + 1]);
    if (q != wg) load_grad(pa);
    // the next pair of this group: its gradient rows into L2 while this one
    // runs (at 1024^2 and above the mixed fields do not stay in L2 between
    // the column pass and the row pass)
    if (q + W < npair) {
      const int pn = p0 + 2 * (q + W);
      if (product_heavy(L.pk[pn])) {
        const char* a = reinterpret_cast<const char*>(mix + (long long)L.pa[pn] * g.mi + rowoff);
        const char* b = reinterpret_cast<const char*>(mix + (long long)L.pb[pn] * g.mi + rowoff);
        const int bytes = (g.K + 1) * (int)sizeof(cplx<T>);
        for (int off = j * 128; off < bytes; off += G * 128) {
          asm volatile("prefetch.global.L2 [%0];" ::"l"(a + off));
          asm volatile("prefetch.global.L2 [%0];" ::"l"(b + off));
        }
      }
    }
    if (s2) {
      // both products' gathers, issued together ahead of the transforms
      gather(pa, S0);
      if (h2) gather(pa + 1, S1);
    }
    if (product_heavy(L.pk[pa])) gfft<T, +1, L_, SYNC, false>(x, buf0, buf1, w, j, gi, d.tw);
    form(pa, 0, S0);
    if (h2) {
      // the second product needs its own transform: park the first
#pragma unroll
      for (int m = 0; m < 8; ++m) P0[m * G + j] = x[m].x;
      load_grad(pa + 1);
      gfft<T, +1, L_, SYNC, false>(x, buf0, buf1, w, j, gi, d.tw);
      form(pa + 1, 1, S1);
#pragma unroll
      for (int m = 0; m < 8; ++m) x[m].x = P0[m * G + j];
    } else if (npq == 2) {
      form(pa + 1, 1, nullptr);
    } else {
#pragma unroll
      for (int m = 0; m < 8; ++m) x[m].y = (T)0;
    }
    gfft<T, -1, L_, SYNC, false>(x, buf0, buf1, w, j, gi, d.tw);
    store_pair_spectrum_ct<T, L_, SYNC>(x, buf0, buf1, w, d.pmix + (long long)pa * g.mi,
                                        npq == 2 ? d.pmix + (long long)(pa + 1) * g.mi : nullptr, rowoff, j, gi,
                                        g.K, g.KXP);
  }
  };
  if constexpr (WARP) dispatch_L<4, 8>(d.g.log2N, body);
  else dispatch_L<4, 11>(d.g.log2N, body);
  pdl_release();
}

// ---------------------------------------------------------------------------
// a4 (second half): right-hand sides and RK4 with integrating factor, one
// thread per (evolved field, two modes); local block = (field, mode block).
//   stage 0: a = N(y_n)      acc = E^2 a            y1 = E (y_n + dt/2 a)
//   stage 1: b = N(y1)       acc += 2 E b           y2 = E y_n + dt/2 b
//   stage 2: c = N(y2)       acc += 2 E c           y3 = E^2 y_n + dt E c
//   stage 3: d = N(y3)       y_{n+1} = E^2 y_n + dt/6 (acc + d)
// with E = exp(-nu |k|^2p dt/2) (Heun and forward Euler: see update_mode).
// Stage inputs alternate between two buffers
// (a thread reads other fields' stage inputs at its mode).
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

// Two-dimensional Euler model: the velocity of the vorticity zeta in buffer b
// at mode m, through the streamfunction (lap psi = zeta, u = -d_y psi,
// v = d_x psi): u_hat = i ky zeta_hat/|k|^2, v_hat = -i kx zeta_hat/|k|^2, zero
// at k = 0; written beside zeta.
template <typename T>
__device__ __forceinline__ void slave_velocity(cplx<T>* b, const Layout& L, long long ms, long long m, T kxf, T kyf) {
  const cplx<T> z = b[L.f_h * ms + m];
  const T k2 = kxf * kxf + kyf * kyf;
  const T inv = k2 > (T)0 ? (T)1 / k2 : (T)0;
  b[L.f_u * ms + m] = mk<T>(-kyf * z.y * inv, kyf * z.x * inv);
  b[L.f_v * ms + m] = mk<T>(kxf * z.y * inv, -kxf * z.x * inv);
}

// y_{n+1} = E^2 y_n + inc at element o of field f, with the factor E^2 given
// as the unevaluated sum e2h + e2l (the part e2l y_n joins the increment);
// compensated in FP32 for the fields marked so.
template <typename T>
__device__ __forceinline__ void commit_mode(const RunDesc<T>& d, int f, long long o, T e2h, T e2l, cplx<T> inc) {
  const cplx<T> yn = d.y[o];
  inc.x = fma(yn.x, e2l, inc.x);
  inc.y = fma(yn.y, e2l, inc.y);
  if (d.comp && d.L.fkahan[f]) {
    cplx<T> cc = d.comp[o];
    cc.x *= e2h;
    cc.y *= e2h;
    cplx<T> out;
    out.x = kahan_add_rn(yn.x * e2h, inc.x, cc.x);
    out.y = kahan_add_rn(yn.y * e2h, inc.y, cc.y);
    d.y[o] = out;
    d.comp[o] = cc;
  } else {
    d.y[o] = mk<T>(fma(yn.x, e2h, inc.x), fma(yn.y, e2h, inc.y));
  }
}

// Right-hand side and RK4 update of evolved field f at mode m = kyi*KXP + kx
// (kx <= K); prod(p) returns the spectral product p at this mode.
template <typename T, typename PF>
__device__ __forceinline__ void update_mode(const RunDesc<T>& d, int stage, T sd, bool even, int f, int m,
                                            int kx, int kyi, PF prod) {
  const Geom& g = d.g;
  const Layout& L = d.L;
  const int st = d.c.stepper;
  const int msi = (int)g.ms;
  const int role = L.frole[f], slot = L.fslot[f];
  // two-dimensional Euler model: u and v follow zeta (written with it)
  const bool e2 = L.model == 2;
  if (e2 && (role == R_U || role == R_V)) return;
  const int cls = L.fclass[f];
  const T E = cls == IF_NONE ? (T)1 : d.ef[3 * cls * msi + m];
  // E^2 = e2h + e2l for the commit of y_{n+1} (read where it is committed)
  auto e2h = [&]() { return cls == IF_NONE ? (T)1 : d.ef[(3 * cls + 1) * msi + m]; };
  auto e2l = [&]() { return cls == IF_NONE ? (T)0 : d.ef[(3 * cls + 2) * msi + m]; };
  const int o = f * msi + m;
  const T kxf = (T)kx, kyf = (T)(kyi - g.K);
  // xi-first scheme (Strategy 2, forward Euler): xi steps by 2 dt on even
  // steps, gbar on odd ones (integrating factor over 2 dt: E^4)
  const bool x1 = L.scheme == SCHEME_XI_FIRST && (role == R_P || role == R_G);
  const bool active = !x1 || ((role == R_P) == even);
  if (!active) return;
  if (st == 2 && stage == 1) {
    // forward Euler, second pass: y_{n+1} = E^2 y_n + dt E^2 a, the increment
    // from the first pass (a separate pass: the first reads other fields' y_n)
    const T h2 = e2h(), l2 = e2l();
    if (x1) {
      // E^4 = (h2 + l2)^2 to the same precision (exact product of h2 by fma)
      const T e4h = h2 * h2;
      const T e4l = fma(h2, h2, -e4h) + (T)2 * h2 * l2;
      commit_mode<T>(d, f, o, e4h, e4l, d.acc[o]);
    } else {
      commit_mode<T>(d, f, o, h2, l2, d.acc[o]);
    }
    if (e2 && role == R_H) slave_velocity<T>(d.y, L, g.ms, m, kxf, kyf);
    return;
  }
  const T dt = d.cdt;
  const cplx<T>* yin = stage_input(d, stage);
  cplx<T> rhs;
  if (role <= R_H) {
    // shallow-water right-hand side, Eq. (sw_eqs_dimless)
    if (e2) {
      // vorticity of the two-dimensional Euler flow: d_t zeta = -div(u zeta)
      rhs = csub<T>(mk<T>(0, 0), cadd<T>(cik<T>(prod(L.p_zu), kxf), cik<T>(prod(L.p_zv), kyf)));
    } else if (L.model == 0) {
      if (role == R_H) {
        rhs = csub<T>(mk<T>(0, 0), cadd<T>(cik<T>(prod(L.p_hu), kxf), cik<T>(prod(L.p_hv), kyf)));
      } else {
        const cplx<T> hh = yin[L.f_h * msi + m];
        const cplx<T> Bq = cadd<T>(cscale<T>(hh, d.cc2), prod(L.p_ke));
        if (role == R_U)
          rhs = csub<T>(cadd<T>(cscale<T>(yin[L.f_v * msi + m], d.cf0), prod(L.p_zv)), cik<T>(Bq, kxf));
        else
          rhs = csub<T>(csub<T>(cscale<T>(yin[L.f_u * msi + m], -d.cf0), prod(L.p_zu)), cik<T>(Bq, kyf));
      }
    } else {
      const T kc = kxf * d.cadvx + kyf * d.cadvy;
      rhs = cik<T>(yin[f * msi + m], -kc);
    }
  } else if (role == R_P) {
    const cplx<T> pp = prod(L.p_p[slot]);
    if (L.strategy == 1) {
      // d_t D = s u - u.grad D
      cplx<T> ua;
      if (L.model == 1) {
        const bool k0 = (kx == 0 && kyi == g.K);
        ua = mk<T>(k0 ? (slot == 0 ? d.cadvx : d.cadvy) : (T)0, 0);
      } else {
        ua = yin[(slot == 0 ? L.f_u : L.f_v) * msi + m];
      }
      rhs = csub<T>(cscale<T>(ua, (T)sd), pp);
    } else {
      rhs = pp;  // xi: the product holds u(x+xi) - w - w.grad xi
    }
  } else {
    // f_hat of the averaged scalar at this stage
    const int sc = L.lmf[slot];
    cplx<T> fh;
    if (sc == LMF_ZETA)
      fh = e2 ? yin[L.f_h * msi + m]  // the evolved vorticity (its mean included)
              : csub<T>(cik<T>(yin[L.f_v * msi + m], kxf), cik<T>(yin[L.f_u * msi + m], kyf));
    else if (sc == LMF_H) fh = yin[L.f_h * msi + m];
    else if (sc == LMF_U) fh = yin[L.f_u * msi + m];
    else if (sc == LMF_V) fh = yin[L.f_v * msi + m];
    else fh = prod(L.p_q);
    if (role == R_E) {
      rhs = fh;  // Eq. (ave)
    } else {
      const cplx<T> pg = prod(L.p_g[slot]);
      // S1: f - u.grad g (Eq. gtilde-evol); S2: f(x+xi) - w.grad g
      rhs = L.strategy == 1 ? csub<T>(fh, pg) : pg;
    }
  }
  const cplx<T> yn = d.y[o];
  cplx<T>* yout = stage == 1 ? d.ysb : d.ysa;
  const bool last = stage == stage_count(st) - 1;
  if (st == 2) {
    // forward Euler, first pass: the increment dt E^2 a (xi-first mean
    // fields: 2 dt E^4 a)
    d.acc[o] = cscale<T>(rhs, x1 ? (T)2 * dt * (E * E) * (E * E) : dt * E * E);
  } else if (!last && st != 0) {
    // Heun, stage 0: acc = E^2 a, y1 = E^2 (y_n + dt a)
    d.acc[o] = cscale<T>(rhs, E * E);
    yout[o] = cscale<T>(cadd<T>(yn, cscale<T>(rhs, dt)), E * E);
  } else if (stage == 0 && !last) {
    d.acc[o] = cscale<T>(rhs, E * E);
    yout[o] = cscale<T>(cadd<T>(yn, cscale<T>(rhs, (T)0.5 * dt)), E);
  } else if (stage == 1 && !last) {
    d.acc[o] = cadd<T>(d.acc[o], cscale<T>(rhs, (T)2 * E));
    yout[o] = cadd<T>(cscale<T>(yn, E), cscale<T>(rhs, (T)0.5 * dt));
  } else if (stage == 2) {
    d.acc[o] = cadd<T>(d.acc[o], cscale<T>(rhs, (T)2 * E));
    yout[o] = cadd<T>(cscale<T>(yn, E * E), cscale<T>(rhs, dt * E));
  } else {
    // final stage: y_{n+1} = E^2 y_n + inc, with inc = dt/6 (acc + d) (RK4)
    // or dt/2 (acc + b) (Heun); its inputs are the stage buffers, not y
    commit_mode<T>(d, f, o, e2h(), e2l(), cscale<T>(cadd<T>(d.acc[o], rhs), st == 0 ? dt / (T)6 : dt / (T)2));
  }
  if (e2 && role == R_H && st != 2) slave_velocity<T>(last ? d.y : yout, L, g.ms, m, kxf, kyf);
}

// Modes per block of the update kernel: 512 (two per thread: the grid of a
// 256^2 Strategy-1 + Strategy-2 batch then fits in one wave of blocks, with
// six resident blocks per SM in FP32, i.e. at most 40 registers) up to
// 512^2; 2048 (eight per thread) from 1024^2, where the larger blocks
// amortise their set-up (7% faster at 2048^2, twice slower at 256^2).
constexpr int UPD_MODES = 512;
__host__ __device__ __forceinline__ int update_modes(int N) { return N >= 1024 ? 2048 : UPD_MODES; }
template <typename T> constexpr int update_min_blocks() { return sizeof(T) == 4 ? 6 : 4; }

template <typename T>
__global__ void __launch_bounds__(256, update_min_blocks<T>()) k_stage_update(const RunDesc<T>* __restrict__ runs,
                                                      const int* __restrict__ start, int nruns, int stage) {
  const int r = find_run(start, nruns, blockIdx.x);
  LM_STAGE_DESC(T);  // many field lookups per thread: read from shared memory
  pdl_wait();  // state written by the previous kernels: only after this
  const Geom& g = d.g;
  const Layout& L = d.L;
  const int lb = blockIdx.x - start[r];
  const int upm = update_modes(g.N);
  const int mblocks = (int)((g.ms + upm - 1) / upm);
  const int f = lb / mblocks;
  const long long m0 = (long long)(lb - f * mblocks) * upm + threadIdx.x;
  const T sd = stage_time<T>(d.ctr, stage, d.cdt, d.c.stepper);
  const bool even = L.scheme == SCHEME_XI_FIRST ? ((*d.ctr & 1LL) == 0) : true;
  auto modes = [&](auto Uc) {
    constexpr int NU = decltype(Uc)::value;
    // element offsets of a run fit in 32 bits (16 fields x 933,465 modes at
    // 2048^2); the mode's (ky, kx) advance by 256 modes per step without a
    // division each
    const int msi = (int)g.ms, KXP = g.KXP;
    int mi = (int)m0;
    int kyi = mi / KXP, kx = mi - kyi * KXP;
    const int dq = 256 / KXP, dr = 256 - dq * KXP;
#pragma unroll
    for (int u = 0; u < NU; ++u) {
      if (mi < msi && kx <= g.K) {
        const int mm = mi;
        update_mode<T>(d, stage, sd, even, f, mm, kx, kyi, [&](int p) { return d.ps[p * msi + mm]; });
      }
      mi += 256;
      kx += dr;
      kyi += dq;
      if (kx >= KXP) {
        kx -= KXP;
        ++kyi;
      }
    }
  };
  if (upm == UPD_MODES) modes(IntC<UPD_MODES / 256>());
  else modes(IntC<2048 / 256>());
  if (stage == stage_count(d.c.stepper) - 1) {
    // the run's last block to finish advances its step counter (every block
    // of the run has read it above, before taking its ticket)
    __syncthreads();
    if (threadIdx.x == 0) {
      __threadfence();
      const unsigned t = atomicAdd(d.ticket, 1u);
      if (t == (unsigned)d.nb[KT_UPDATE] - 1u) {
        *d.ticket = 0u;
        *d.ctr = *d.ctr + 1;
        __threadfence();
      }
    }
  }
  pdl_release();
}

}  // namespace lm
