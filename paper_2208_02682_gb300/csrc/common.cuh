// common.cuh -- types, data layout and kernel parameter blocks shared by the
// GB300 kernels of the Lagrangian-mean shallow-water library.
//
// Data layout in HBM (all complex arrays interleaved re/im):
//   spectral field  : [ky_idx][kx], ky_idx = ky + K in [0, 2K], kx in [0, KXP)
//                     (K = floor((N-1)/3) is the 2/3-rule cutoff; KXP is K+1
//                     rounded up to a multiple of 4; columns kx > K are zero)
//   column-transformed intermediate ("mixed" field, physical y, spectral kx):
//                     [y][kx], y in [0, N), kx in [0, KXP)
//   physical field  : [y][x] real, row-major.
// The mixed layout is written by the column pass with 4-wide kx tiles and read
// by the row pass row by row, so both sides access 32-byte (FP32) or 64-byte
// (FP64) contiguous runs.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

namespace lm {

template <typename T> struct CT;
template <> struct CT<float> { typedef float2 type; };
template <> struct CT<double> { typedef double2 type; };
template <typename T> using cplx = typename CT<T>::type;

template <typename T> __host__ __device__ __forceinline__ cplx<T> mk(T x, T y) {
  cplx<T> r; r.x = x; r.y = y; return r;
}
template <typename T> __device__ __forceinline__ cplx<T> cadd(cplx<T> a, cplx<T> b) { return mk<T>(a.x + b.x, a.y + b.y); }
template <typename T> __device__ __forceinline__ cplx<T> csub(cplx<T> a, cplx<T> b) { return mk<T>(a.x - b.x, a.y - b.y); }
template <typename T> __device__ __forceinline__ cplx<T> cmul(cplx<T> a, cplx<T> b) {
  return mk<T>(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x);
}
template <typename T> __device__ __forceinline__ cplx<T> cscale(cplx<T> a, T s) { return mk<T>(a.x * s, a.y * s); }
template <typename T> __device__ __forceinline__ cplx<T> cconj(cplx<T> a) { return mk<T>(a.x, -a.y); }
// multiply by i*k (spectral derivative)
template <typename T> __device__ __forceinline__ cplx<T> cik(cplx<T> a, T k) { return mk<T>(-a.y * k, a.x * k); }

// Shared-memory position of element n of a transform: one spare slot every
// 8 elements.  Shared memory serves 8-byte accesses per half-warp from 16
// slots of 8 bytes (16-byte accesses per quarter-warp from 8 slots); the
// padding spreads the stride-8 writes of the first radix-8 pass over
// distinct slots.  (An XOR swizzle that also keeps the consecutive accesses
// conflict-free halves the shared-memory wavefronts of the FFT kernels but
// costs more index arithmetic than it saves: the kernels are bound by
// latency, not by shared-memory bandwidth.)
template <typename T>
__host__ __device__ __forceinline__ int sidx(int n) {
  return n + (n >> 3);
}
// Distance between the transforms of a block (rows, or the columns of a
// column tile).
template <typename T>
__host__ __device__ __forceinline__ int row_stride(int N) { return N + (N >> 3); }
template <typename T>
__host__ __device__ __forceinline__ int col_stride(int N, int C) { return N + (N >> 3); }
// Column tiles on group transforms (lanes interleave the C columns): each
// column owns two exchange buffers, and successive columns are offset by a
// number of slots (16 for FP32, 8 for FP64, per bank row) congruent to
// slots/C, so the C lanes that share a row index use distinct slots.
template <typename T>
__host__ __device__ __forceinline__ int col_buf_stride(int N, int C) {
  const int S = sizeof(T) == 4 ? 16 : 8;
  const int st = 2 * (N + (N >> 3));
  const int tgt = C <= S ? S / C : 1;
  return st + (((tgt - st) % S) + S) % S;
}

// ---------------------------------------------------------------------------
// Geometry of one grid
struct Geom {
  int N, log2N, K, KX, KXP, NY;
  long long ms;  // complex elements per spectral field  (NY * KXP)
  long long mi;  // complex elements per mixed field     (N * KXP)
  long long np;  // reals per physical field             (N * N)
};

// ---------------------------------------------------------------------------
// Field bookkeeping for one configuration (strategy, mask) of a handle.
enum { MAXF = 16, MAXI = 24, MAXP = 16 };
enum { OP_ID = 0, OP_DX = 1, OP_DY = 2, OP_CURL = 3 };
enum { LMF_ZETA = 0, LMF_H = 1, LMF_U = 2, LMF_V = 3, LMF_Q = 4, NLMF = 5 };
// physical fields of the row pass (and of the Strategy-2 gather buffer)
enum { PH_U = 0, PH_V = 1, PH_H = 2, PH_Z = 3, PH_Q = 4, PH_XX = 5, PH_XY = 6, NPH = 7 };
// products formed in physical space by the row pass
enum {
  PK_ZV = 0,   // zeta v
  PK_ZU = 1,   // zeta u
  PK_KE = 2,   // (u^2 + v^2)/2
  PK_HU = 3,   // h u
  PK_HV = 4,   // h v
  PK_Q = 5,    // (f0 + zeta)/h
  PK_ADV = 6,  // u d_x G + v d_y G            (Strategy 1; a, b: mixed d_x G, d_y G)
  PK_XI = 7,   // u_c(x+xi) - w_c - w.grad xi_c (Strategy 2; c: component)
  PK_GBAR = 8  // f(x+xi) - w.grad g           (Strategy 2; c: PH_* of f)
};
// integrating-factor classes
enum { IF_DYN = 0, IF_LM = 1, IF_NONE = 2 };
// role of an evolved field in the right-hand side
enum { R_U = 0, R_V = 1, R_H = 2, R_G = 3, R_P = 4, R_E = 5 };

struct Layout {
  int strategy;   // 0: dynamics only, 1 or 2
  int scheme;     // SCHEME_* (the C ABI's LM_SCHEME_*) of the open interval
  int model;      // 0 shallow water, 1 kinematic
  int nf;         // evolved spectral fields
  int ni;         // mixed intermediates produced by the column pass
  int np;         // product fields produced by the row pass
  int nlm;        // number of Lagrangian-mean scalar fields
  int lmf[NLMF];  // which scalar (LMF_*) each LM slot averages
  int has_pos, eulerian, has_q;
  // evolved-field indices
  int f_u, f_v, f_h;
  int f_g[NLMF];     // g~ (S1) or gbar (S2) per LM slot
  int f_p[2];        // D (S1) or xi (S2) components
  int f_e[NLMF];     // Eulerian accumulators per LM slot
  int fclass[MAXF];  // IF_* class of each evolved field
  int fkahan[MAXF];  // compensated final update (FP32 mode) for this field
  int frole[MAXF];   // R_* role
  int fslot[MAXF];   // LM slot (R_G, R_E) or component (R_P)
  // column pass: output i = op(src[i] (, src2[i]))
  int i_src[MAXI], i_src2[MAXI], i_op[MAXI];
  int i_u, i_v, i_h, i_z;      // dynamics intermediates
  int i_xi[2];                 // xi components (Strategy 2)
  // row pass: product list
  int pk[MAXP], pa[MAXP], pb[MAXP], pc[MAXP];
  // product index feeding each right-hand side (-1: none)
  int p_zv, p_zu, p_ke, p_hu, p_hv, p_q;
  int p_g[NLMF];
  int p_p[2];
  // some pair (2q, 2q+1) of the row pass has a second product that needs a
  // transform or gather of its own (only when the products are not all
  // paired heavy-with-light, e.g. the kinematic model)
  int heavy2;
  int pad_;
};

// discretisation of the mean equations (the C ABI's LM_SCHEME_* values)
enum { SCHEME_COUPLED = 0, SCHEME_XI_FIRST = 1 };

struct StepConsts {
  double dt, f0, c2, adv_x, adv_y;
  int stepper;  // SW_STEP_* (0 RK4, 1 Heun, 2 forward Euler)
  int pad;
};

// Programmatic dependent launch (PTX griddepcontrol).  The stage kernels of
// a step are launched with programmatic stream serialisation, so a kernel's
// blocks may start while the previous kernel of the stream finishes.
// pdl_wait: before its first access to memory that earlier kernels write,
// a stage kernel waits until they have completed and their writes are
// visible (without the launch attribute it returns at once).  pdl_release:
// after its last store, the kernel lets the next one be scheduled.
__device__ __forceinline__ void pdl_wait() { asm volatile("griddepcontrol.wait;" ::: "memory"); }
__device__ __forceinline__ void pdl_release() { asm volatile("griddepcontrol.launch_dependents;" ::: "memory"); }

// passes of the stage pipeline per step of a stepper: RK4 4 stages, Heun 2,
// forward Euler 1 stage and an update-only pass that commits y_{n+1}
__host__ __device__ __forceinline__ int stage_count(int stepper) { return stepper == 0 ? 4 : 2; }

}  // namespace lm
