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
// a1: column inverse pass, local block = (output field, kx tile).
template <typename T>
__global__ void __launch_bounds__(1024) k_stage_col_inv(const RunDesc<T>* __restrict__ runs,
                                                        const int* __restrict__ start, int nruns, int stage) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const int r = find_run(start, nruns, blockIdx.x);
  const RunDesc<T>& d = runs[r];
  const int lb = blockIdx.x - start[r];
  const int ntile = d.g.KXP >> d.lC;
  const int o = lb / ntile, tile = lb - o * ntile;
  const cplx<T>* src = stage_input(d, stage);
  const int s1 = d.L.i_src[o], s2 = d.L.i_src2[o] < 0 ? s1 : d.L.i_src2[o];
  col_inverse_tile<T>(reinterpret_cast<cplx<T>*>(smem_raw), src + (long long)s1 * d.g.ms,
                      src + (long long)s2 * d.g.ms, d.L.i_op[o], d.mix + (long long)o * d.g.mi, d.g, d.lC,
                      tile << d.lC, d.tw);
}

// a4 (first half): column forward pass of the products, local block =
// (product, kx tile).
template <typename T>
__global__ void __launch_bounds__(1024) k_stage_col_fwd(const RunDesc<T>* __restrict__ runs,
                                                        const int* __restrict__ start, int nruns) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const int r = find_run(start, nruns, blockIdx.x);
  const RunDesc<T>& d = runs[r];
  const int lb = blockIdx.x - start[r];
  const int ntile = d.g.KXP >> d.lC;
  const int p = lb / ntile, tile = lb - p * ntile;
  col_forward_tile<T>(reinterpret_cast<cplx<T>*>(smem_raw), d.pmix + (long long)p * d.g.mi,
                      d.ps + (long long)p * d.g.ms, d.g, d.lC, tile << d.lC, d.tw);
}

// a3: Strategy-2 gather buffer (physical u, v | h, zeta), local block =
// (pair, row block).
template <typename T>
__global__ void __launch_bounds__(256) k_stage_row_inv(const RunDesc<T>* __restrict__ runs,
                                                       const int* __restrict__ start, int nruns) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  cplx<T>* buf = reinterpret_cast<cplx<T>*>(smem_raw);
  const int r = find_run(start, nruns, blockIdx.x);
  const RunDesc<T>& d = runs[r];
  const Geom& g = d.g;
  const int lb = blockIdx.x - start[r];
  const int nrb = g.N / d.Bi;
  const int pair = lb / nrb, rb = lb - pair * nrb;
  const int B = d.Bi, N = g.N, row0 = rb * B;
  const int ia = pair == 0 ? d.L.i_u : d.L.i_h, ib = pair == 0 ? d.L.i_v : d.L.i_z;
  const int oa = pair == 0 ? PH_U : PH_H, ob = pair == 0 ? PH_V : PH_Z;
  row_pair_inverse<T>(buf, d.mix + (long long)ia * g.mi, d.mix + (long long)ib * g.mi, row0, B, g, d.tw);
  for (int e = threadIdx.x; e < B * N; e += blockDim.x) {
    const int rr = e >> g.log2N, x = e & (N - 1);
    const cplx<T> v = buf[rr * pad8(N) + pad8(x)];
    const long long off = (long long)(row0 + rr) * N + x;
    d.phys[oa * g.np + off] = v.x;
    d.phys[ob * g.np + off] = v.y;
  }
}

// q = (f0 + zeta)/h, h = 1 + eta, into the gather buffer (Strategy 2 with PV
// averaged).
template <typename T>
__global__ void __launch_bounds__(256) k_stage_phys_q(const RunDesc<T>* __restrict__ runs,
                                                      const int* __restrict__ start, int nruns) {
  const int r = find_run(start, nruns, blockIdx.x);
  const RunDesc<T>& d = runs[r];
  const long long i = (long long)(blockIdx.x - start[r]) * blockDim.x + threadIdx.x;
  const long long np = d.g.np;
  if (i < np) d.phys[PH_Q * np + i] = ((T)d.c.f0 + d.phys[PH_Z * np + i]) / ((T)1 + d.phys[PH_H * np + i]);
}

// ---------------------------------------------------------------------------
// a2: row pass with products.  Local block = (pair group, row block): Bp rows
// and product pairs [grp*ppb, (grp+1)*ppb).  Smem: W, P (Bp*pad8(N) complex
// each), U (4*Bp*N reals: u, v, h, zeta), XI (2*Bp*N reals, Strategy 2).
template <typename T>
__global__ void __launch_bounds__(256) k_stage_row_prod(const RunDesc<T>* __restrict__ runs,
                                                        const int* __restrict__ start, int nruns, int stage) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const int r = find_run(start, nruns, blockIdx.x);
  const RunDesc<T>& d = runs[r];
  const Geom& g = d.g;
  const Layout& L = d.L;
  const int N = g.N, B = d.Bp;
  const int bst = pad8(N);
  const int lb = blockIdx.x - start[r];
  const int nrb = N / B;
  const int grp = lb / nrb, rb = lb - grp * nrb;
  cplx<T>* W = reinterpret_cast<cplx<T>*>(smem_raw);
  cplx<T>* P = W + B * bst;
  T* U = reinterpret_cast<T*>(P + B * bst);
  T* XI = U + 4 * B * N;
  const int row0 = rb * B;
  const int np = L.np;
  const int p0 = grp * d.ppb * 2;
  const int p1 = min(np, p0 + d.ppb * 2);
  const int nthr = blockDim.x, tid = threadIdx.x;
  const int BN = B * N;
  const bool kin = L.model == 1;
  const T adv_x = (T)d.c.adv_x, adv_y = (T)d.c.adv_y;
  const T f0 = (T)d.c.f0;
  const double s = stage_time(d.ctr, stage, d.c.dt);
  const bool s0 = !(s > 0.0);
  const T inv_s = s0 ? (T)0 : (T)(1.0 / s);
  const T inv_dx = (T)((double)N / 6.283185307179586476925286766559);
  const cplx<T>* mix = d.mix;

  // which physical base fields this block's products read
  bool need_uv = false, need_hz = false;
  for (int p = p0; p < p1; ++p) {
    const int k = L.pk[p];
    if (k == PK_ZV || k == PK_ZU || k == PK_HU || k == PK_HV || k == PK_Q) need_hz = true;
    if (k == PK_ZV || k == PK_ZU || k == PK_KE || k == PK_HU || k == PK_HV) need_uv = true;
    if ((k == PK_ADV || k == PK_XI || k == PK_GBAR) && !kin) need_uv = true;
  }
  // physical u, v, h, zeta (and xi) of the block's rows
  if (L.strategy == 2) {
    for (int e = tid; e < BN; e += nthr) {
      const long long off = (long long)row0 * N + e;
#pragma unroll
      for (int f = 0; f < 4; ++f) U[f * BN + e] = d.phys[f * g.np + off];
    }
    row_pair_inverse<T>(W, mix + (long long)L.i_xi[0] * g.mi, mix + (long long)L.i_xi[1] * g.mi, row0, B, g,
                        d.tw);
    for (int e = tid; e < BN; e += nthr) {
      const int rr = e >> g.log2N, x = e & (N - 1);
      const cplx<T> v = W[rr * bst + pad8(x)];
      XI[e] = v.x;
      XI[BN + e] = v.y;
    }
  } else {
    if (need_uv) {
      row_pair_inverse<T>(W, mix + (long long)L.i_u * g.mi, mix + (long long)L.i_v * g.mi, row0, B, g, d.tw);
      for (int e = tid; e < BN; e += nthr) {
        const int rr = e >> g.log2N, x = e & (N - 1);
        const cplx<T> v = W[rr * bst + pad8(x)];
        U[e] = v.x;
        U[BN + e] = v.y;
      }
      __syncthreads();
    }
    if (need_hz) {
      row_pair_inverse<T>(W, mix + (long long)L.i_h * g.mi, mix + (long long)L.i_z * g.mi, row0, B, g, d.tw);
      for (int e = tid; e < BN; e += nthr) {
        const int rr = e >> g.log2N, x = e & (N - 1);
        const cplx<T> v = W[rr * bst + pad8(x)];
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
    if (need_grad)
      row_pair_inverse<T>(W, mix + (long long)L.pa[p] * g.mi, mix + (long long)L.pb[p] * g.mi, row0, B, g, d.tw);
    const int pc = L.pc[p];
    for (int e = tid; e < BN; e += nthr) {
      const int rr = e >> g.log2N, x = e & (N - 1);
      const T u = U[e], v = U[BN + e], h = U[2 * BN + e], z = U[3 * BN + e];
      T val;
      switch (kind) {
        case PK_ZV: val = z * v; break;
        case PK_ZU: val = z * u; break;
        case PK_KE: val = (T)0.5 * (u * u + v * v); break;
        // depth h = 1 + eta; the state and the row buffers hold eta
        case PK_HU: val = u + h * u; break;
        case PK_HV: val = v + h * v; break;
        case PK_Q: val = (f0 + z) / ((T)1 + h); break;
        case PK_ADV: {
          // u.grad G (Eq. gtilde-evol) or u.grad D
          const cplx<T> dd = W[rr * bst + pad8(x)];
          const T ua = kin ? adv_x : u, va = kin ? adv_y : v;
          val = ua * dd.x + va * dd.y;
          break;
        }
        default: {
          // Strategy 2, Eqs. (xi_evol), (barf_xi): w = xi/s, limit u/2 at s = 0
          const cplx<T> dd = W[rr * bst + pad8(x)];
          const T xx = XI[e], xy = XI[BN + e];
          const T ua = kin ? adv_x : u, va = kin ? adv_y : v;
          const T wx = s0 ? (T)0.5 * ua : xx * inv_s;
          const T wy = s0 ? (T)0.5 * va : xy * inv_s;
          const T wg = wx * dd.x + wy * dd.y;
          const int yy = row0 + rr;
          if (kind == PK_XI) {
            T ui;
            if (kin) ui = pc == 0 ? adv_x : adv_y;
            else ui = bilinear<T>(d.phys + (long long)pc * g.np, x, yy, xx, xy, inv_dx, N);
            val = ui - (pc == 0 ? wx : wy) - wg;
          } else {
            const T fi = bilinear<T>(d.phys + (long long)pc * g.np, x, yy, xx, xy, inv_dx, N);
            val = fi - wg;
          }
          break;
        }
      }
      cplx<T>& dst = P[rr * bst + pad8(x)];
      if (slot == 0) dst = mk<T>(val, (T)0);
      else dst.y = val;
    }
    if (slot == 0) {
      pend = p;
      slot = 1;
    } else {
      row_pair_forward_store<T>(P, d.pmix + (long long)pend * g.mi, d.pmix + (long long)p * g.mi, row0, B, g,
                                d.tw);
      slot = 0;
    }
    __syncthreads();
  }
  if (slot == 1) row_pair_forward_store<T>(P, d.pmix + (long long)pend * g.mi, nullptr, row0, B, g, d.tw);
}

// ---------------------------------------------------------------------------
// a4 (second half): right-hand sides and RK4 with integrating factor, one
// thread per (mode, evolved field); local block = (field, mode block).
//   stage 0: a = N(y_n)      acc = E^2 a            y1 = E (y_n + dt/2 a)
//   stage 1: b = N(y1)       acc += 2 E b           y2 = E y_n + dt/2 b
//   stage 2: c = N(y2)       acc += 2 E c           y3 = E^2 y_n + dt E c
//   stage 3: d = N(y3)       y_{n+1} = E^2 y_n + dt/6 (acc + d)
// with E = exp(-nu |k|^8 dt/2).  Stage inputs alternate between two buffers
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

template <typename T>
__global__ void __launch_bounds__(256) k_stage_update(const RunDesc<T>* __restrict__ runs,
                                                      const int* __restrict__ start, int nruns, int stage) {
  const int r = find_run(start, nruns, blockIdx.x);
  LM_STAGE_DESC(T);  // many field lookups per thread: read from shared memory
  const Geom& g = d.g;
  const Layout& L = d.L;
  const int lb = blockIdx.x - start[r];
  const int mblocks = (int)((g.ms + 255) / 256);
  const int f = lb / mblocks;
  const long long m = (long long)(lb - f * mblocks) * 256 + threadIdx.x;
  const double sd = stage_time(d.ctr, stage, d.c.dt);
  if (m < g.ms) {
    const int kyi = (int)(m / g.KXP), kx = (int)(m - (long long)kyi * g.KXP);
    if (kx <= g.K) {
      const T kxf = (T)kx, kyf = (T)(kyi - g.K);
      const T dt = (T)d.c.dt;
      const cplx<T>* yin = stage_input(d, stage);
      const cplx<T>* ps = d.ps;
      const int role = L.frole[f], slot = L.fslot[f];
      cplx<T> rhs;
      if (role <= R_H) {
        // shallow-water right-hand side, Eq. (sw_eqs_dimless)
        if (L.model == 0) {
          if (role == R_H) {
            rhs = csub<T>(mk<T>(0, 0), cadd<T>(cik<T>(ps[L.p_hu * g.ms + m], kxf), cik<T>(ps[L.p_hv * g.ms + m], kyf)));
          } else {
            const cplx<T> hh = yin[L.f_h * g.ms + m];
            const cplx<T> Bq = cadd<T>(cscale<T>(hh, (T)d.c.c2), ps[L.p_ke * g.ms + m]);
            if (role == R_U)
              rhs = csub<T>(cadd<T>(cscale<T>(yin[L.f_v * g.ms + m], (T)d.c.f0), ps[L.p_zv * g.ms + m]), cik<T>(Bq, kxf));
            else
              rhs = csub<T>(csub<T>(cscale<T>(yin[L.f_u * g.ms + m], -(T)d.c.f0), ps[L.p_zu * g.ms + m]), cik<T>(Bq, kyf));
          }
        } else {
          const T kc = kxf * (T)d.c.adv_x + kyf * (T)d.c.adv_y;
          rhs = cik<T>(yin[f * g.ms + m], -kc);
        }
      } else if (role == R_P) {
        const cplx<T> pp = ps[L.p_p[slot] * g.ms + m];
        if (L.strategy == 1) {
          // d_t D = s u - u.grad D
          cplx<T> ua;
          if (L.model == 1) {
            const bool k0 = (kx == 0 && kyi == g.K);
            ua = mk<T>(k0 ? (T)(slot == 0 ? d.c.adv_x : d.c.adv_y) : (T)0, 0);
          } else {
            ua = yin[(slot == 0 ? L.f_u : L.f_v) * g.ms + m];
          }
          rhs = csub<T>(cscale<T>(ua, (T)sd), pp);
        } else {
          rhs = pp;  // xi: the product holds u(x+xi) - w - w.grad xi
        }
      } else {
        // f_hat of the averaged scalar at this stage
        const int sc = L.lmf[slot];
        cplx<T> fh;
        if (sc == LMF_ZETA) fh = csub<T>(cik<T>(yin[L.f_v * g.ms + m], kxf), cik<T>(yin[L.f_u * g.ms + m], kyf));
        else if (sc == LMF_H) fh = yin[L.f_h * g.ms + m];
        else if (sc == LMF_U) fh = yin[L.f_u * g.ms + m];
        else if (sc == LMF_V) fh = yin[L.f_v * g.ms + m];
        else fh = ps[L.p_q * g.ms + m];
        if (role == R_E) {
          rhs = fh;  // Eq. (ave)
        } else {
          const cplx<T> pg = ps[L.p_g[slot] * g.ms + m];
          // S1: f - u.grad g (Eq. gtilde-evol); S2: f(x+xi) - w.grad g
          rhs = L.strategy == 1 ? csub<T>(fh, pg) : pg;
        }
      }
      const int cls = L.fclass[f];
      const T E = cls == IF_NONE ? (T)1 : d.ef[cls * g.ms + m];
      const long long o = f * g.ms + m;
      const cplx<T> yn = d.y[o];
      cplx<T>* yout = stage == 1 ? d.ysb : d.ysa;
      if (stage == 0) {
        d.acc[o] = cscale<T>(rhs, E * E);
        yout[o] = cscale<T>(cadd<T>(yn, cscale<T>(rhs, (T)0.5 * dt)), E);
      } else if (stage == 1) {
        d.acc[o] = cadd<T>(d.acc[o], cscale<T>(rhs, (T)2 * E));
        yout[o] = cadd<T>(cscale<T>(yn, E), cscale<T>(rhs, (T)0.5 * dt));
      } else if (stage == 2) {
        d.acc[o] = cadd<T>(d.acc[o], cscale<T>(rhs, (T)2 * E));
        yout[o] = cadd<T>(cscale<T>(yn, E * E), cscale<T>(rhs, dt * E));
      } else {
        const cplx<T> inc = cscale<T>(cadd<T>(d.acc[o], rhs), dt / (T)6);
        const T E2 = E * E;
        if (d.comp && L.fkahan[f]) {
          cplx<T> cc = d.comp[o];
          cc.x *= E2;
          cc.y *= E2;
          cplx<T> out;
          out.x = kahan_add_rn(yn.x * E2, inc.x, cc.x);
          out.y = kahan_add_rn(yn.y * E2, inc.y, cc.y);
          d.y[o] = out;
          d.comp[o] = cc;
        } else {
          d.y[o] = cadd<T>(cscale<T>(yn, E2), inc);
        }
      }
    }
  }
  if (stage == 3) {
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
}

}  // namespace lm
