// lagmean.cu -- C ABI (include/lagmean.h): handles, field layout, the RK4
// stage pipeline replayed from a captured CUDA graph, and the FP64 transforms
// around it (initial condition, end-of-interval means, diagnostics).
#include <cuda_runtime.h>

#include <cmath>
#include <cstdio>
#include <cstring>
#include <new>
#include <string>

#include "../../include/lagmean.h"
#include "launch.cuh"

using namespace lm;

namespace lm {
cudaError_t prepare_kernels_f32();
cudaError_t prepare_kernels_f64();
}  // namespace lm

static thread_local std::string g_create_error;

namespace lm {
// message for calls without a handle (sw_create, sw_project_static)
void set_handleless_error(const std::string& msg) { g_create_error = msg; }
}  // namespace lm

struct sw_handle {
  sw_params p;
  Geom g;
  cudaStream_t stream = nullptr;
  cudaStream_t cap_stream = nullptr;  // private stream used only for graph capture
  bool fp32 = false;
  size_t tsz = 8;  // sizeof(T)
  std::string err;
  // device memory
  void* arena = nullptr;
  size_t arena_bytes = 0;
  void *y = nullptr, *ys = nullptr, *ys2 = nullptr, *acc = nullptr, *comp = nullptr, *ps = nullptr;
  void *mix = nullptr, *pmix = nullptr, *phys = nullptr, *ef = nullptr, *tw = nullptr;
  double2 *tw64 = nullptr, *spec64 = nullptr, *mix64 = nullptr;
  double *out64 = nullptr, *part = nullptr, *dres = nullptr;
  long long* ctr = nullptr;
  unsigned* ticket = nullptr;
  int diag_blocks = 0;
  // interval state
  bool lm_open = false;
  lm_params lp{};
  int64_t done = 0;
  int64_t steps_total = 0;
  Layout L{};
  // captured graphs of 1 and GRAPH_STEPS RK4 steps for the current layout
  cudaGraphExec_t gexec = nullptr;
  cudaGraphExec_t gexec_multi = nullptr;
  bool graph_valid = false;
  int64_t kernels_per_step = 0;
  int64_t launches = 0;  // kernels launched since creation
  // launch shape of the row pass (rows per block, product pairs per block)
  int rows_prod = 1, ppb = 1, rows_inv = 1;
};

static int fail(sw_handle* h, int code, const std::string& msg) {
  if (h) h->err = msg;
  else g_create_error = msg;
  return code;
}
static int fail_cuda(sw_handle* h, const char* what, cudaError_t e) {
  return fail(h, SW_ECUDA, std::string(what) + ": " + cudaGetErrorString(e));
}
#define CK(h, ...)                                                  \
  do {                                                              \
    cudaError_t e_ = (__VA_ARGS__);                                 \
    if (e_ != cudaSuccess) return fail_cuda(h, #__VA_ARGS__, e_);   \
  } while (0)

// ---------------------------------------------------------------------------
// Field layout of a configuration.
static Layout build_layout(int model, int strategy, int fields, int eulerian) {
  Layout L;
  std::memset(&L, 0, sizeof(L));
  L.strategy = strategy;
  L.model = model;
  L.p_zv = L.p_zu = L.p_ke = L.p_hu = L.p_hv = L.p_q = -1;
  for (int j = 0; j < NLMF; ++j) L.f_g[j] = L.f_e[j] = L.p_g[j] = -1;
  L.f_p[0] = L.f_p[1] = L.p_p[0] = L.p_p[1] = L.i_xi[0] = L.i_xi[1] = -1;
  int nf = 0;
  L.f_u = nf++;
  L.f_v = nf++;
  L.f_h = nf++;
  for (int f = 0; f < 3; ++f) {
    L.fclass[f] = IF_DYN;
    L.fkahan[f] = 0;
    L.frole[f] = R_U + f;
    L.fslot[f] = 0;
  }
  if (strategy > 0) {
    const int bits[NLMF] = {LM_ZETA, LM_H, LM_U, LM_V, LM_Q};
    for (int j = 0; j < NLMF; ++j)
      if (fields & bits[j]) L.lmf[L.nlm++] = j;
    L.has_q = (fields & LM_Q) ? 1 : 0;
    L.has_pos = (strategy == 2 || (fields & LM_POS)) ? 1 : 0;
    L.eulerian = eulerian ? 1 : 0;
    auto addf = [&](int cls, int role, int slot) {
      L.fclass[nf] = cls;
      L.fkahan[nf] = 1;
      L.frole[nf] = role;
      L.fslot[nf] = slot;
      return nf++;
    };
    for (int j = 0; j < L.nlm; ++j) L.f_g[j] = addf(IF_LM, R_G, j);
    if (L.has_pos)
      for (int c = 0; c < 2; ++c) L.f_p[c] = addf(IF_LM, R_P, c);
    if (L.eulerian)
      for (int j = 0; j < L.nlm; ++j) L.f_e[j] = addf(IF_NONE, R_E, j);
  }
  L.nf = nf;
  // column-pass outputs
  int ni = 0;
  auto addi = [&](int src, int op, int src2) {
    L.i_src[ni] = src;
    L.i_op[ni] = op;
    L.i_src2[ni] = src2;
    return ni++;
  };
  L.i_u = addi(L.f_u, OP_ID, -1);
  L.i_v = addi(L.f_v, OP_ID, -1);
  L.i_h = addi(L.f_h, OP_ID, -1);
  L.i_z = addi(L.f_u, OP_CURL, L.f_v);
  // products
  int np = 0;
  auto addp = [&](int kind, int a, int b, int c) {
    L.pk[np] = kind;
    L.pa[np] = a;
    L.pb[np] = b;
    L.pc[np] = c;
    return np++;
  };
  if (model == SW_MODEL_SW) {
    L.p_zv = addp(PK_ZV, -1, -1, 0);
    L.p_zu = addp(PK_ZU, -1, -1, 0);
    L.p_ke = addp(PK_KE, -1, -1, 0);
    L.p_hu = addp(PK_HU, -1, -1, 0);
    L.p_hv = addp(PK_HV, -1, -1, 0);
  }
  if (L.has_q) L.p_q = addp(PK_Q, -1, -1, 0);
  const int ph_of[NLMF] = {PH_Z, PH_H, PH_U, PH_V, PH_Q};
  if (strategy == 1) {
    for (int j = 0; j < L.nlm; ++j) {
      const int gx = addi(L.f_g[j], OP_DX, -1), gy = addi(L.f_g[j], OP_DY, -1);
      L.p_g[j] = addp(PK_ADV, gx, gy, 0);
    }
    if (L.has_pos)
      for (int c = 0; c < 2; ++c) {
        const int dx = addi(L.f_p[c], OP_DX, -1), dy = addi(L.f_p[c], OP_DY, -1);
        L.p_p[c] = addp(PK_ADV, dx, dy, 0);
      }
  } else if (strategy == 2) {
    L.i_xi[0] = addi(L.f_p[0], OP_ID, -1);
    L.i_xi[1] = addi(L.f_p[1], OP_ID, -1);
    for (int c = 0; c < 2; ++c) {
      const int dx = addi(L.f_p[c], OP_DX, -1), dy = addi(L.f_p[c], OP_DY, -1);
      L.p_p[c] = addp(PK_XI, dx, dy, c);
    }
    for (int j = 0; j < L.nlm; ++j) {
      const int gx = addi(L.f_g[j], OP_DX, -1), gy = addi(L.f_g[j], OP_DY, -1);
      L.p_g[j] = addp(PK_GBAR, gx, gy, ph_of[L.lmf[j]]);
    }
  }
  L.ni = ni;
  L.np = np;
  return L;
}

// ---------------------------------------------------------------------------
// Algorithmic bytes of one launch of each stepping kernel: the distinct input
// elements it must read and the output elements it must write (box modes
// NY*KX, mixed rows N*KX, physical N*N), not counting L2 hits or padding.
struct KBytes {
  double col_inv, row_inv, phys_q, row_prod, col_fwd, update[4];
};

static KBytes kernel_bytes(const sw_handle* h, const Layout& L) {
  const Geom& g = h->g;
  const double cs = 2.0 * h->tsz, ts = (double)h->tsz;
  const double MB = (double)g.NY * g.KX, MI = (double)g.N * g.KX, NP = (double)g.np;
  KBytes b;
  bool seen[MAXF] = {};
  int nsrc = 0;
  for (int i = 0; i < L.ni; ++i) {
    if (!seen[L.i_src[i]]) { seen[L.i_src[i]] = true; ++nsrc; }
    if (L.i_src2[i] >= 0 && !seen[L.i_src2[i]]) { seen[L.i_src2[i]] = true; ++nsrc; }
  }
  b.col_inv = nsrc * MB * cs + L.ni * MI * cs;
  b.row_inv = 4 * MI * cs + 4 * NP * ts;
  b.phys_q = 3 * NP * ts;
  double rp = L.np * MI * cs;
  if (L.strategy == 2) {
    bool gat[NPH] = {};
    int ng = 0;
    for (int p = 0; p < L.np; ++p) {
      int f = -1;
      if (L.pk[p] == PK_XI && L.model == 0) f = L.pc[p];
      if (L.pk[p] == PK_GBAR) f = L.pc[p];
      if (f >= 0 && !gat[f]) { gat[f] = true; ++ng; }
    }
    rp += (L.ni - 4) * MI * cs + 4 * NP * ts + ng * NP * ts;
  } else {
    rp += L.ni * MI * cs;
  }
  b.row_prod = rp;
  b.col_fwd = L.np * (MI + MB) * cs;
  int nk = 0;
  for (int f = 0; f < L.nf; ++f) nk += L.fkahan[f];
  const double nf = L.nf, np = L.np;
  b.update[0] = (nf + np + 2 * nf) * MB * cs + 2 * MB * ts;
  b.update[1] = b.update[2] = (3 * nf + np + 2 * nf) * MB * cs + 2 * MB * ts;
  b.update[3] = (3 * nf + np + nf + (h->fp32 ? 2 * nk : 0)) * MB * cs + 2 * MB * ts;
  return b;
}

// Optional per-launch event bracketing (sw_kernel_times).
struct Prof {
  enum { MAXEV = 64 };
  cudaEvent_t ev[2 * MAXEV];
  int cls[MAXEV];
  double bytes[MAXEV];
  int n = 0;
};

#define LAUNCH(cls_, bytes_, ...)                                    \
  do {                                                               \
    if (pf) cudaEventRecord(pf->ev[2 * pf->n], s);                   \
    if ((e = (__VA_ARGS__)) != cudaSuccess) return e;                \
    if (pf) {                                                        \
      cudaEventRecord(pf->ev[2 * pf->n + 1], s);                     \
      pf->cls[pf->n] = (cls_);                                       \
      pf->bytes[pf->n] = (bytes_);                                   \
      pf->n++;                                                       \
    }                                                                \
    ++*nlaunch;                                                      \
  } while (0)

// ---------------------------------------------------------------------------
// Stage pipeline (one RK4 step = 4 stages) for precision T.
template <typename T>
static cudaError_t enqueue_step(sw_handle* h, cudaStream_t s, Prof* pf, int64_t* nlaunch) {
  const Layout& L = h->L;
  const Geom& g = h->g;
  const KBytes kb = kernel_bytes(h, L);
  cplx<T>* y = (cplx<T>*)h->y;
  // stage inputs: stage 1 and 3 read ysa, stage 2 reads ysb
  cplx<T>* ysa = (cplx<T>*)h->ys;
  cplx<T>* ysb = (cplx<T>*)h->ys2;
  StepConsts c{h->p.dt, h->p.f0, h->p.c2, h->p.adv_x, h->p.adv_y};
  cudaError_t e;
  for (int stage = 0; stage < 4; ++stage) {
    const cplx<T>* src = stage == 0 ? y : (stage == 2 ? ysb : ysa);
    cplx<T>* dst_next = (stage == 1) ? ysb : ysa;
    if (L.np > 0) {
      ColInvArgs<T> ci;
      ci.src = src;
      ci.dst = (cplx<T>*)h->mix;
      ci.tw = (const cplx<T>*)h->tw;
      ci.g = g;
      ci.nout = L.ni;
      for (int i = 0; i < L.ni; ++i) {
        ci.src_idx[i] = L.i_src[i];
        ci.src2_idx[i] = L.i_src2[i];
        ci.op[i] = L.i_op[i];
        ci.dst_idx[i] = i;
      }
      LAUNCH(SW_K_COL_INV, kb.col_inv, launch_col_inv<T>(ci, s));
      if (L.strategy == 2) {
        RowInvArgs<T, T> ri;
        std::memset(&ri, 0, sizeof(ri));
        ri.src = (const cplx<T>*)h->mix;
        ri.dst = (T*)h->phys;
        ri.dst_stride = g.np;
        ri.tw = (const cplx<T>*)h->tw;
        ri.g = g;
        ri.B = h->rows_inv;
        ri.npairs = 2;
        ri.a_idx[0] = L.i_u; ri.b_idx[0] = L.i_v; ri.oa[0] = PH_U; ri.ob[0] = PH_V;
        ri.a_idx[1] = L.i_h; ri.b_idx[1] = L.i_z; ri.oa[1] = PH_H; ri.ob[1] = PH_Z;
        for (int p = 0; p < 2; ++p) ri.sa[p] = ri.sb[p] = 1.0;
        LAUNCH(SW_K_ROW_INV, kb.row_inv, launch_row_inv<T, T>(ri, s));
        if (L.has_q) LAUNCH(SW_K_PHYS_Q, kb.phys_q, launch_phys_q<T>((T*)h->phys, g.np, h->p.f0, s));
      }
      RowProdArgs<T> rp;
      rp.mix = (const cplx<T>*)h->mix;
      rp.prod = (cplx<T>*)h->pmix;
      rp.phys = (const T*)h->phys;
      rp.ctr = h->ctr;
      rp.tw = (const cplx<T>*)h->tw;
      rp.g = g;
      rp.L = L;
      rp.c = c;
      rp.B = h->rows_prod;
      rp.ppb = h->ppb;
      rp.stage = stage;
      LAUNCH(SW_K_ROW_PROD, kb.row_prod, launch_row_prod<T>(rp, s));
      ColFwdArgs<T> cf;
      cf.src = (const cplx<T>*)h->pmix;
      cf.dst = (cplx<T>*)h->ps;
      cf.tw = (const cplx<T>*)h->tw;
      cf.g = g;
      cf.nout = L.np;
      for (int i = 0; i < L.np; ++i) cf.src_idx[i] = cf.dst_idx[i] = i;
      LAUNCH(SW_K_COL_FWD, kb.col_fwd, launch_col_fwd<T>(cf, s));
    }
    UpdateArgs<T> ua;
    ua.y = y;
    ua.ysin = src;
    ua.ys = dst_next;
    ua.acc = (cplx<T>*)h->acc;
    ua.comp = h->fp32 ? (cplx<T>*)h->comp : nullptr;
    ua.ps = (const cplx<T>*)h->ps;
    ua.ef = (const T*)h->ef;
    ua.ctr = h->ctr;
    ua.ticket = h->ticket;
    ua.g = g;
    ua.L = L;
    ua.c = c;
    ua.stage = stage;
    LAUNCH(SW_K_UPDATE, kb.update[stage], launch_update<T>(ua, s));
  }
  return cudaSuccess;
}

static const int GRAPH_STEPS = 8;

static void drop_graph(sw_handle* h) {
  if (h->gexec) cudaGraphExecDestroy(h->gexec);
  if (h->gexec_multi) cudaGraphExecDestroy(h->gexec_multi);
  h->gexec = h->gexec_multi = nullptr;
  h->graph_valid = false;
}

// Capture `steps` RK4 steps into an executable graph.  Capture runs on a
// private stream (the caller's stream may be the legacy default stream, which
// cannot be captured); the graphs are launched on the caller's stream.
static int capture_steps(sw_handle* h, int steps, cudaGraphExec_t* out) {
  cudaGraph_t graph = nullptr;
  if (!h->cap_stream) CK(h, cudaStreamCreateWithFlags(&h->cap_stream, cudaStreamNonBlocking));
  CK(h, cudaStreamBeginCapture(h->cap_stream, cudaStreamCaptureModeThreadLocal));
  int64_t nl = 0;
  cudaError_t e = cudaSuccess;
  for (int i = 0; i < steps && e == cudaSuccess; ++i)
    e = h->fp32 ? enqueue_step<float>(h, h->cap_stream, nullptr, &nl)
                : enqueue_step<double>(h, h->cap_stream, nullptr, &nl);
  cudaError_t e2 = cudaStreamEndCapture(h->cap_stream, &graph);
  if (e != cudaSuccess) {
    if (graph) cudaGraphDestroy(graph);
    return fail_cuda(h, "enqueue_step (capture)", e);
  }
  if (e2 != cudaSuccess) return fail_cuda(h, "cudaStreamEndCapture", e2);
  e = cudaGraphInstantiate(out, graph, 0);
  cudaGraphDestroy(graph);
  if (e != cudaSuccess) {
    *out = nullptr;
    return fail_cuda(h, "cudaGraphInstantiate", e);
  }
  h->kernels_per_step = nl / steps;
  return SW_OK;
}

static int ensure_graph(sw_handle* h) {
  if (h->graph_valid) return SW_OK;
  drop_graph(h);
  int rc = capture_steps(h, 1, &h->gexec);
  if (rc == SW_OK) rc = capture_steps(h, GRAPH_STEPS, &h->gexec_multi);
  if (rc != SW_OK) {
    drop_graph(h);
    return rc;
  }
  h->graph_valid = true;
  return SW_OK;
}

static int run_steps(sw_handle* h, int64_t n) {
  if (n <= 0) return SW_OK;
  int rc = ensure_graph(h);
  if (rc) return rc;
  int64_t i = 0;
  for (; i + GRAPH_STEPS <= n; i += GRAPH_STEPS) CK(h, cudaGraphLaunch(h->gexec_multi, h->stream));
  for (; i < n; ++i) CK(h, cudaGraphLaunch(h->gexec, h->stream));
  h->steps_total += n;
  h->launches += n * h->kernels_per_step;
  return SW_OK;
}

// ---------------------------------------------------------------------------
// FP64 transforms around the stepping.

// Physical FP64 fields (N*N each, in h->out64[slot..]) from up to two
// spectral fields of the state: value = (y - comp)*scale, plus ax*x + ay*y.
struct OutSpec {
  int field;  // evolved-field index (-1: none)
  double scale, ax, ay;
  int slot;   // output slot in out64
};

static int spectral_pair_to_phys(sw_handle* h, const OutSpec& a, const OutSpec* b) {
  const Geom& g = h->g;
  cudaStream_t s = h->stream;
  // FP64 spectral copies (scale applied in the row pass epilogue)
  if (h->fp32)
    CK(h, launch_spec_to_f64<float>((const cplx<float>*)h->y, (const cplx<float>*)h->comp, h->spec64, g.ms,
                                    a.field, b ? b->field : -1, 1.0, s));
  else
    CK(h, launch_spec_to_f64<double>((const cplx<double>*)h->y, nullptr, h->spec64, g.ms, a.field,
                                     b ? b->field : -1, 1.0, s));
  ColInvArgs<double> ci;
  ci.src = h->spec64;
  ci.dst = h->mix64;
  ci.tw = h->tw64;
  ci.g = g;
  ci.nout = b ? 2 : 1;
  for (int i = 0; i < 2; ++i) {
    ci.src_idx[i] = i;
    ci.src2_idx[i] = -1;
    ci.op[i] = OP_ID;
    ci.dst_idx[i] = i;
  }
  CK(h, launch_col_inv<double>(ci, s));
  RowInvArgs<double, double> ri;
  std::memset(&ri, 0, sizeof(ri));
  ri.src = h->mix64;
  ri.dst = h->out64;
  ri.dst_stride = g.np;
  ri.tw = h->tw64;
  ri.g = g;
  ri.B = h->rows_inv;
  ri.npairs = 1;
  ri.a_idx[0] = 0;
  ri.b_idx[0] = b ? 1 : -1;
  ri.oa[0] = a.slot;
  ri.ob[0] = b ? b->slot : -1;
  ri.sa[0] = a.scale;
  ri.axa[0] = a.ax;
  ri.aya[0] = a.ay;
  if (b) {
    ri.sb[0] = b->scale;
    ri.axb[0] = b->ax;
    ri.ayb[0] = b->ay;
  }
  CK(h, launch_row_inv<double, double>(ri, s));
  h->launches += 3;
  return SW_OK;
}

static int phys_outputs(sw_handle* h, const OutSpec* os, int n) {
  for (int i = 0; i < n; i += 2) {
    int rc = spectral_pair_to_phys(h, os[i], i + 1 < n ? &os[i + 1] : nullptr);
    if (rc) return rc;
  }
  return SW_OK;
}

// Load a physical FP64 initial condition (already in out64[0..2]) into the
// dynamics fields of the state.
static int load_ic_from_out64(sw_handle* h) {
  const Geom& g = h->g;
  cudaStream_t s = h->stream;
  RowFwdArgs<double> rf;
  std::memset(&rf, 0, sizeof(rf));
  rf.src = h->out64;
  rf.dst = h->mix64;
  rf.tw = h->tw64;
  rf.g = g;
  rf.B = h->rows_inv;
  rf.npairs = 2;
  rf.a_idx[0] = 0; rf.b_idx[0] = 1; rf.oa[0] = 0; rf.ob[0] = 1;
  rf.a_idx[1] = 2; rf.b_idx[1] = -1; rf.oa[1] = 2; rf.ob[1] = -1;
  CK(h, launch_row_fwd<double>(rf, s));
  ColFwdArgs<double> cf;
  cf.src = h->mix64;
  cf.dst = h->spec64;
  cf.tw = h->tw64;
  cf.g = g;
  cf.nout = 3;
  for (int i = 0; i < 3; ++i) cf.src_idx[i] = cf.dst_idx[i] = i;
  CK(h, launch_col_fwd<double>(cf, s));
  if (h->fp32) CK(h, launch_spec_from_f64<float>(h->spec64, (cplx<float>*)h->y, 3 * g.ms, s));
  else CK(h, launch_spec_from_f64<double>(h->spec64, (cplx<double>*)h->y, 3 * g.ms, s));
  h->launches += 3;
  return SW_OK;
}

static int copy_in_uvh(sw_handle* h, const double* uvh, int on_device) {
  const size_t bytes = (size_t)3 * h->g.np * sizeof(double);
  CK(h, cudaMemcpyAsync(h->out64, uvh, bytes, on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice,
                        h->stream));
  return load_ic_from_out64(h);
}

// ---------------------------------------------------------------------------
static bool is_pow2(int n) { return n > 0 && (n & (n - 1)) == 0; }

static int validate(const sw_params* p, std::string& why) {
  if (!p) { why = "params is NULL"; return SW_EINVAL; }
  if (!is_pow2(p->N) || p->N < 16 || p->N > 2048) { why = "N must be a power of two in [16, 2048]"; return SW_EINVAL; }
  if (p->precision != SW_PREC_FP64 && p->precision != SW_PREC_FP32) { why = "precision must be SW_PREC_FP64 or SW_PREC_FP32"; return SW_EINVAL; }
  if (p->model != SW_MODEL_SW && p->model != SW_MODEL_KINEMATIC) { why = "model must be SW_MODEL_SW or SW_MODEL_KINEMATIC"; return SW_EINVAL; }
  if (p->reserved != 0) { why = "reserved must be 0"; return SW_EINVAL; }
  if (!(p->dt > 0.0) || !std::isfinite(p->dt)) { why = "dt must be finite and > 0"; return SW_EINVAL; }
  if (!std::isfinite(p->f0) || !std::isfinite(p->adv_x) || !std::isfinite(p->adv_y)) { why = "f0 and adv must be finite"; return SW_EINVAL; }
  if (!(p->c2 >= 0.0) || !std::isfinite(p->c2)) { why = "c2 must be finite and >= 0"; return SW_EINVAL; }
  if (!(p->nu8 >= 0.0) || !(p->lm_nu8 >= 0.0) || !std::isfinite(p->nu8) || !std::isfinite(p->lm_nu8)) { why = "nu8, lm_nu8 must be finite and >= 0"; return SW_EINVAL; }
  return SW_OK;
}

static size_t align256(size_t x) { return (x + 255) & ~(size_t)255; }

template <typename T>
static void host_tables(const sw_params& p, const Geom& g, void* ef_host, void* tw_host, double2* tw64_host) {
  T* ef = (T*)ef_host;
  cplx<T>* tw = (cplx<T>*)tw_host;
  for (int kyi = 0; kyi < g.NY; ++kyi)
    for (int kx = 0; kx < g.KXP; ++kx) {
      const double ky = kyi - g.K;
      const double k2 = (double)kx * kx + ky * ky;
      const double k8 = k2 * k2 * k2 * k2;
      const long long m = (long long)kyi * g.KXP + kx;
      ef[m] = (T)std::exp(-p.nu8 * k8 * p.dt * 0.5);
      ef[g.ms + m] = (T)std::exp(-p.lm_nu8 * k8 * p.dt * 0.5);
    }
  const double twopi = 6.283185307179586476925286766559;
  for (int t = 0; t < g.N; ++t) {
    const double a = twopi * (double)t / (double)g.N;
    tw64_host[t] = make_double2(std::cos(a), -std::sin(a));
    tw[t] = mk<T>((T)std::cos(a), (T)(-std::sin(a)));
  }
}

extern "C" int sw_create(const sw_params* p, const double* ic_uvh, int ic_on_device, void* stream,
                         sw_handle** out) {
  g_create_error.clear();
  if (!out) return fail(nullptr, SW_EINVAL, "out is NULL");
  *out = nullptr;
  std::string why;
  int rc = validate(p, why);
  if (rc) return fail(nullptr, rc, why);
  if (!ic_uvh) return fail(nullptr, SW_EINVAL, "ic_uvh is NULL");
  static bool prepared = false;
  if (!prepared) {
    cudaError_t e = prepare_kernels_f32();
    if (e == cudaSuccess) e = prepare_kernels_f64();
    if (e != cudaSuccess) return fail(nullptr, SW_ECUDA, std::string("kernel set-up: ") + cudaGetErrorString(e));
    prepared = true;
  }
  sw_handle* h = new (std::nothrow) sw_handle();
  if (!h) return fail(nullptr, SW_ENOMEM, "host allocation failed");
  h->p = *p;
  h->stream = (cudaStream_t)stream;
  h->fp32 = p->precision == SW_PREC_FP32;
  h->tsz = h->fp32 ? 4 : 8;
  Geom& g = h->g;
  g.N = p->N;
  g.log2N = 0;
  while ((1 << g.log2N) < g.N) ++g.log2N;
  g.K = (g.N - 1) / 3;
  g.KX = g.K + 1;
  g.KXP = (g.KX + 3) / 4 * 4;
  g.NY = 2 * g.K + 1;
  g.ms = (long long)g.NY * g.KXP;
  g.mi = (long long)g.N * g.KXP;
  g.np = (long long)g.N * g.N;
  const size_t cs = 2 * h->tsz;  // complex T
  h->diag_blocks = 1024;
  h->rows_prod = row_block_rows(g.N);
  h->rows_inv = row_block_rows(g.N);
  h->ppb = g.N <= 512 ? 1 : MAXP;
  // arena layout
  size_t off = 0;
  auto take = [&](size_t bytes) { size_t o = off; off += align256(bytes); return o; };
  const size_t o_y = take(MAXF * g.ms * cs), o_ys = take(MAXF * g.ms * cs), o_ys2 = take(MAXF * g.ms * cs);
  const size_t o_acc = take(MAXF * g.ms * cs);
  const size_t o_comp = take(MAXF * g.ms * cs), o_ps = take(MAXP * g.ms * cs);
  const size_t o_mix = take(MAXI * g.mi * cs), o_pmix = take(MAXP * g.mi * cs);
  const size_t o_phys = take(NPH * g.np * h->tsz), o_ef = take(2 * g.ms * h->tsz), o_tw = take(g.N * cs);
  const size_t o_tw64 = take(g.N * sizeof(double2)), o_spec64 = take(4 * g.ms * sizeof(double2));
  const size_t o_mix64 = take(4 * g.mi * sizeof(double2)), o_out64 = take(12 * g.np * sizeof(double));
  const size_t o_part = take(2 * h->diag_blocks * sizeof(double)), o_dres = take(4 * sizeof(double));
  const size_t o_ctr = take(sizeof(long long)), o_ticket = take(sizeof(unsigned));
  h->arena_bytes = off;
  cudaError_t e = cudaMalloc(&h->arena, h->arena_bytes);
  if (e != cudaSuccess) {
    delete h;
    cudaGetLastError();
    return fail(nullptr, SW_ENOMEM, std::string("cudaMalloc: ") + cudaGetErrorString(e));
  }
  char* base = (char*)h->arena;
  h->y = base + o_y; h->ys = base + o_ys; h->ys2 = base + o_ys2; h->acc = base + o_acc; h->comp = base + o_comp; h->ps = base + o_ps;
  h->mix = base + o_mix; h->pmix = base + o_pmix; h->phys = base + o_phys; h->ef = base + o_ef;
  h->tw = base + o_tw; h->tw64 = (double2*)(base + o_tw64); h->spec64 = (double2*)(base + o_spec64);
  h->mix64 = (double2*)(base + o_mix64); h->out64 = (double*)(base + o_out64);
  h->part = (double*)(base + o_part); h->dres = (double*)(base + o_dres);
  h->ctr = (long long*)(base + o_ctr); h->ticket = (unsigned*)(base + o_ticket);
  // tables
  const size_t ef_bytes = 2 * g.ms * h->tsz, tw_bytes = g.N * cs;
  char* hbuf = (char*)std::malloc(ef_bytes + tw_bytes + g.N * sizeof(double2));
  if (!hbuf) {
    cudaFree(h->arena);
    delete h;
    return fail(nullptr, SW_ENOMEM, "host allocation failed");
  }
  if (h->fp32) host_tables<float>(*p, g, hbuf, hbuf + ef_bytes, (double2*)(hbuf + ef_bytes + tw_bytes));
  else host_tables<double>(*p, g, hbuf, hbuf + ef_bytes, (double2*)(hbuf + ef_bytes + tw_bytes));
  rc = SW_OK;
  do {
    if ((e = cudaMemsetAsync(h->arena, 0, h->arena_bytes, h->stream)) != cudaSuccess) break;
    if ((e = cudaMemcpyAsync(h->ef, hbuf, ef_bytes, cudaMemcpyHostToDevice, h->stream)) != cudaSuccess) break;
    if ((e = cudaMemcpyAsync(h->tw, hbuf + ef_bytes, tw_bytes, cudaMemcpyHostToDevice, h->stream)) != cudaSuccess) break;
    if ((e = cudaMemcpyAsync(h->tw64, hbuf + ef_bytes + tw_bytes, g.N * sizeof(double2), cudaMemcpyHostToDevice,
                             h->stream)) != cudaSuccess) break;
    if ((e = cudaStreamSynchronize(h->stream)) != cudaSuccess) break;
  } while (0);
  std::free(hbuf);
  if (e != cudaSuccess) {
    std::string m = std::string("device set-up: ") + cudaGetErrorString(e);
    cudaFree(h->arena);
    delete h;
    return fail(nullptr, SW_ECUDA, m);
  }
  h->L = build_layout(p->model, 0, 0, 0);
  rc = copy_in_uvh(h, ic_uvh, ic_on_device);
  if (rc == SW_OK) {
    e = cudaStreamSynchronize(h->stream);
    if (e != cudaSuccess) rc = fail_cuda(h, "initial transform", e);
  }
  if (rc != SW_OK) {
    std::string m = h->err;
    cudaFree(h->arena);
    delete h;
    return fail(nullptr, rc, m);
  }
  *out = h;
  return SW_OK;
}

extern "C" void sw_destroy(sw_handle* h) {
  if (!h) return;
  cudaStreamSynchronize(h->stream);
  drop_graph(h);
  if (h->cap_stream) cudaStreamDestroy(h->cap_stream);
  if (h->arena) cudaFree(h->arena);
  delete h;
}

extern "C" int sw_step(sw_handle* h, int64_t nsteps) {
  if (!h) return SW_EINVAL;
  h->err.clear();
  if (nsteps < 0) return fail(h, SW_EINVAL, "nsteps < 0");
  if (h->lm_open) return fail(h, SW_EBUSY, "an averaging interval is open");
  return run_steps(h, nsteps);
}

extern "C" int lmean_begin(sw_handle* h, const lm_params* lp) {
  if (!h) return SW_EINVAL;
  h->err.clear();
  if (!lp) return fail(h, SW_EINVAL, "lm_params is NULL");
  if (h->lm_open) return fail(h, SW_ESTATE, "an averaging interval is already open");
  if (lp->strategy != 1 && lp->strategy != 2) return fail(h, SW_EINVAL, "strategy must be 1 or 2");
  if (lp->reserved != 0) return fail(h, SW_EINVAL, "reserved must be 0");
  if (lp->n_steps < 1) return fail(h, SW_EINVAL, "n_steps must be >= 1");
  if (lp->fields & ~(LM_ZETA | LM_H | LM_U | LM_V | LM_Q | LM_POS))
    return fail(h, SW_EINVAL, "unknown bits in fields");
  const int scal = lp->fields & (LM_ZETA | LM_H | LM_U | LM_V | LM_Q);
  if (!scal && !(lp->fields & LM_POS)) return fail(h, SW_EINVAL, "no field selected");
  if (!scal && lp->eulerian) return fail(h, SW_EINVAL, "Eulerian means need a scalar field");
  Layout L = build_layout(h->p.model, lp->strategy, lp->fields, lp->eulerian);
  const Geom& g = h->g;
  const size_t cs = 2 * h->tsz;
  // zero the mean fields, their compensation terms and the step counter
  CK(h, cudaMemsetAsync((char*)h->y + 3 * g.ms * cs, 0, (size_t)(MAXF - 3) * g.ms * cs, h->stream));
  CK(h, cudaMemsetAsync(h->comp, 0, (size_t)MAXF * g.ms * cs, h->stream));
  CK(h, cudaMemsetAsync(h->ctr, 0, sizeof(long long), h->stream));
  drop_graph(h);
  h->L = L;
  h->lp = *lp;
  h->done = 0;
  h->lm_open = true;
  return SW_OK;
}

extern "C" int lmean_step(sw_handle* h, int64_t nsteps) {
  if (!h) return SW_EINVAL;
  h->err.clear();
  if (!h->lm_open) return fail(h, SW_ESTATE, "no averaging interval is open");
  if (nsteps < 0) return fail(h, SW_EINVAL, "nsteps < 0");
  if (nsteps > h->lp.n_steps - h->done) return fail(h, SW_ERANGE, "more steps than remain in the interval");
  int rc = run_steps(h, nsteps);
  if (rc == SW_OK) h->done += nsteps;
  return rc;
}

extern "C" int lmean_progress(sw_handle* h, int64_t* done, int64_t* remaining) {
  if (!h) return SW_EINVAL;
  if (done) *done = h->lm_open ? h->done : 0;
  if (remaining) *remaining = h->lm_open ? h->lp.n_steps - h->done : 0;
  return SW_OK;
}

static int copy_out(sw_handle* h, double* dst, int slot, int on_device) {
  if (!dst) return SW_OK;
  const size_t bytes = (size_t)h->g.np * sizeof(double);
  CK(h, cudaMemcpyAsync(dst, h->out64 + (size_t)slot * h->g.np, bytes,
                        on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost, h->stream));
  return SW_OK;
}

extern "C" int lmean_end(sw_handle* h, const lm_result* out) {
  if (!h) return SW_EINVAL;
  h->err.clear();
  if (!h->lm_open) return fail(h, SW_ESTATE, "no averaging interval is open");
  if (h->done != h->lp.n_steps) return fail(h, SW_ESTATE, "interval not complete");
  if (!out) return fail(h, SW_EINVAL, "out is NULL");
  const Layout& L = h->L;
  const double T = (double)h->lp.n_steps * h->p.dt;
  double* lm_ptr[NLMF] = {out->zeta, out->h, out->u, out->v, out->q};
  double* e_ptr[NLMF] = {out->e_zeta, out->e_h, out->e_u, out->e_v, out->e_q};
  bool in_mask[NLMF] = {false, false, false, false, false};
  for (int j = 0; j < L.nlm; ++j) in_mask[L.lmf[j]] = true;
  for (int f = 0; f < NLMF; ++f) {
    if (lm_ptr[f] && !in_mask[f]) return fail(h, SW_EINVAL, "output requested for a field not averaged");
    if (e_ptr[f] && (!in_mask[f] || !L.eulerian)) return fail(h, SW_EINVAL, "Eulerian output not accumulated");
  }
  if ((out->pos_x || out->pos_y) && !L.has_pos) return fail(h, SW_EINVAL, "positions not computed");
  OutSpec os[12];
  double* dst[12];
  int n = 0;
  for (int j = 0; j < L.nlm; ++j)
    if (lm_ptr[L.lmf[j]]) {
      os[n] = OutSpec{L.f_g[j], 1.0 / T, 0.0, 0.0, n};
      dst[n++] = lm_ptr[L.lmf[j]];
    }
  if (L.has_pos) {
    double* pp[2] = {out->pos_x, out->pos_y};
    for (int c = 0; c < 2; ++c)
      if (pp[c]) {
        // S1: Xi^{-1} = x - D/T;  S2: Xi = x + xi
        const double sc = L.strategy == 1 ? -1.0 / T : 1.0;
        os[n] = OutSpec{L.f_p[c], sc, c == 0 ? 1.0 : 0.0, c == 1 ? 1.0 : 0.0, n};
        dst[n++] = pp[c];
      }
  }
  if (L.eulerian)
    for (int j = 0; j < L.nlm; ++j)
      if (e_ptr[L.lmf[j]]) {
        os[n] = OutSpec{L.f_e[j], 1.0 / T, 0.0, 0.0, n};
        dst[n++] = e_ptr[L.lmf[j]];
      }
  int rc = phys_outputs(h, os, n);
  if (rc) return rc;
  for (int i = 0; i < n; ++i)
    if ((rc = copy_out(h, dst[i], i, out->on_device))) return rc;
  if (!out->on_device) CK(h, cudaStreamSynchronize(h->stream));
  h->lm_open = false;
  drop_graph(h);
  h->L = build_layout(h->p.model, 0, 0, 0);
  return SW_OK;
}

extern "C" int sw_get_fields(sw_handle* h, double* uvh, int on_device) {
  if (!h) return SW_EINVAL;
  h->err.clear();
  if (!uvh) return fail(h, SW_EINVAL, "uvh is NULL");
  OutSpec os[3] = {{h->L.f_u, 1.0, 0, 0, 0}, {h->L.f_v, 1.0, 0, 0, 1}, {h->L.f_h, 1.0, 0, 0, 2}};
  // the dynamics fields carry no compensation term (it stays zero)
  int rc = phys_outputs(h, os, 3);
  if (rc) return rc;
  CK(h, cudaMemcpyAsync(uvh, h->out64, (size_t)3 * h->g.np * sizeof(double),
                        on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost, h->stream));
  CK(h, cudaStreamSynchronize(h->stream));
  return SW_OK;
}

extern "C" int sw_set_fields(sw_handle* h, const double* uvh, int on_device) {
  if (!h) return SW_EINVAL;
  h->err.clear();
  if (!uvh) return fail(h, SW_EINVAL, "uvh is NULL");
  if (h->lm_open) return fail(h, SW_EBUSY, "an averaging interval is open");
  int rc = copy_in_uvh(h, uvh, on_device);
  if (rc) return rc;
  CK(h, cudaStreamSynchronize(h->stream));
  return SW_OK;
}

extern "C" int sw_diag(sw_handle* h, double out[3]) {
  if (!h) return SW_EINVAL;
  h->err.clear();
  if (!out) return fail(h, SW_EINVAL, "out is NULL");
  // physical u, v, h, zeta in FP64: zeta via a spectral curl in FP64
  OutSpec os[3] = {{h->L.f_u, 1.0, 0, 0, 0}, {h->L.f_v, 1.0, 0, 0, 1}, {h->L.f_h, 1.0, 0, 0, 2}};
  int rc = phys_outputs(h, os, 3);
  if (rc) return rc;
  // zeta = i kx v - i ky u from FP64 copies of u, v
  const Geom& g = h->g;
  if (h->fp32)
    CK(h, launch_spec_to_f64<float>((const cplx<float>*)h->y, nullptr, h->spec64, g.ms, h->L.f_u, h->L.f_v, 1.0,
                                    h->stream));
  else
    CK(h, launch_spec_to_f64<double>((const cplx<double>*)h->y, nullptr, h->spec64, g.ms, h->L.f_u, h->L.f_v, 1.0,
                                     h->stream));
  ColInvArgs<double> ci;
  ci.src = h->spec64;
  ci.dst = h->mix64;
  ci.tw = h->tw64;
  ci.g = g;
  ci.nout = 1;
  ci.src_idx[0] = 0;
  ci.src2_idx[0] = 1;
  ci.op[0] = OP_CURL;
  ci.dst_idx[0] = 0;
  CK(h, launch_col_inv<double>(ci, h->stream));
  RowInvArgs<double, double> ri;
  std::memset(&ri, 0, sizeof(ri));
  ri.src = h->mix64;
  ri.dst = h->out64;
  ri.dst_stride = g.np;
  ri.tw = h->tw64;
  ri.g = g;
  ri.B = h->rows_inv;
  ri.npairs = 1;
  ri.a_idx[0] = 0;
  ri.b_idx[0] = -1;
  ri.oa[0] = 3;
  ri.ob[0] = -1;
  ri.sa[0] = 1.0;
  CK(h, launch_row_inv<double, double>(ri, h->stream));
  CK(h, launch_diag(h->out64, g.np, h->p.f0, h->p.c2, h->part, h->diag_blocks, h->dres, h->stream));
  h->launches += 5;
  double res[4] = {0, 0, 0, 0};
  CK(h, cudaMemcpyAsync(res, h->dres, 3 * sizeof(double), cudaMemcpyDeviceToHost, h->stream));
  // mass: the k = 0 coefficient of h (row ky = 0, column kx = 0)
  const size_t cs = 2 * h->tsz;
  unsigned char m0[16];
  CK(h, cudaMemcpyAsync(m0, (char*)h->y + ((size_t)h->L.f_h * g.ms + (size_t)g.K * g.KXP) * cs, cs,
                        cudaMemcpyDeviceToHost, h->stream));
  CK(h, cudaStreamSynchronize(h->stream));
  out[0] = h->fp32 ? (double)((float*)m0)[0] : ((double*)m0)[0];
  out[1] = res[1];
  out[2] = res[2];
  return SW_OK;
}

// ---------------------------------------------------------------------------
// Checkpoint blob: header, then the evolved fields and their compensation.
struct BlobHeader {
  char magic[8];
  int32_t version, N, precision, model;
  double dt, f0, c2, nu8, lm_nu8, adv_x, adv_y;
  int32_t lm_open, nf;
  lm_params lp;
  int64_t done, steps_total;
};

static size_t blob_size(sw_handle* h, int nf) {
  return sizeof(BlobHeader) + (size_t)2 * nf * h->g.ms * 2 * h->tsz;
}

extern "C" int sw_get_state(sw_handle* h, void* blob, size_t* size) {
  if (!h) return SW_EINVAL;
  h->err.clear();
  if (!size) return fail(h, SW_EINVAL, "size is NULL");
  const int nf = h->L.nf;
  const size_t need = blob_size(h, nf);
  if (!blob) {
    *size = need;
    return SW_OK;
  }
  if (*size < need) return fail(h, SW_EINVAL, "blob too small");
  BlobHeader hd;
  std::memset(&hd, 0, sizeof(hd));
  std::memcpy(hd.magic, "LAGMEAN1", 8);
  hd.version = 1;
  hd.N = h->p.N; hd.precision = h->p.precision; hd.model = h->p.model;
  hd.dt = h->p.dt; hd.f0 = h->p.f0; hd.c2 = h->p.c2; hd.nu8 = h->p.nu8; hd.lm_nu8 = h->p.lm_nu8;
  hd.adv_x = h->p.adv_x; hd.adv_y = h->p.adv_y;
  hd.lm_open = h->lm_open ? 1 : 0;
  hd.nf = nf;
  hd.lp = h->lp;
  hd.done = h->done;
  hd.steps_total = h->steps_total;
  std::memcpy(blob, &hd, sizeof(hd));
  const size_t fb = (size_t)nf * h->g.ms * 2 * h->tsz;
  char* dst = (char*)blob + sizeof(hd);
  CK(h, cudaMemcpyAsync(dst, h->y, fb, cudaMemcpyDeviceToHost, h->stream));
  CK(h, cudaMemcpyAsync(dst + fb, h->comp, fb, cudaMemcpyDeviceToHost, h->stream));
  CK(h, cudaStreamSynchronize(h->stream));
  *size = need;
  return SW_OK;
}

extern "C" int sw_set_state(sw_handle* h, const void* blob, size_t size) {
  if (!h) return SW_EINVAL;
  h->err.clear();
  if (!blob || size < sizeof(BlobHeader)) return fail(h, SW_EINVAL, "blob too small");
  BlobHeader hd;
  std::memcpy(&hd, blob, sizeof(hd));
  if (std::memcmp(hd.magic, "LAGMEAN1", 8) != 0 || hd.version != 1) return fail(h, SW_EINVAL, "not a state blob");
  if (hd.N != h->p.N || hd.precision != h->p.precision || hd.model != h->p.model || hd.dt != h->p.dt ||
      hd.f0 != h->p.f0 || hd.c2 != h->p.c2 || hd.nu8 != h->p.nu8 || hd.lm_nu8 != h->p.lm_nu8 ||
      hd.adv_x != h->p.adv_x || hd.adv_y != h->p.adv_y)
    return fail(h, SW_EINVAL, "blob parameters differ from the handle's");
  Layout L = hd.lm_open ? build_layout(h->p.model, hd.lp.strategy, hd.lp.fields, hd.lp.eulerian)
                        : build_layout(h->p.model, 0, 0, 0);
  if (L.nf != hd.nf || size < blob_size(h, hd.nf)) return fail(h, SW_EINVAL, "blob size mismatch");
  const size_t fb = (size_t)hd.nf * h->g.ms * 2 * h->tsz;
  const char* src = (const char*)blob + sizeof(hd);
  CK(h, cudaMemcpyAsync(h->y, src, fb, cudaMemcpyHostToDevice, h->stream));
  CK(h, cudaMemcpyAsync(h->comp, src + fb, fb, cudaMemcpyHostToDevice, h->stream));
  long long ctr = hd.done;
  CK(h, cudaMemcpyAsync(h->ctr, &ctr, sizeof(ctr), cudaMemcpyHostToDevice, h->stream));
  CK(h, cudaStreamSynchronize(h->stream));
  drop_graph(h);
  h->L = L;
  h->lm_open = hd.lm_open != 0;
  h->lp = hd.lp;
  h->done = hd.done;
  h->steps_total = hd.steps_total;
  return SW_OK;
}

extern "C" int sw_kernel_times(sw_handle* h, int64_t nsteps, double ms[SW_K_COUNT], int64_t launches[SW_K_COUNT],
                               double bytes[SW_K_COUNT]) {
  if (!h) return SW_EINVAL;
  h->err.clear();
  if (!ms || !launches || !bytes) return fail(h, SW_EINVAL, "output arrays are NULL");
  if (nsteps < 1) return fail(h, SW_EINVAL, "nsteps must be >= 1");
  if (h->lm_open && nsteps > h->lp.n_steps - h->done) return fail(h, SW_ERANGE, "more steps than remain in the interval");
  for (int k = 0; k < SW_K_COUNT; ++k) {
    ms[k] = 0.0;
    launches[k] = 0;
    bytes[k] = 0.0;
  }
  Prof pf;
  int nev = 0;
  cudaError_t e = cudaSuccess;
  for (; nev < 2 * Prof::MAXEV; ++nev)
    if ((e = cudaEventCreate(&pf.ev[nev])) != cudaSuccess) break;
  int rc = SW_OK;
  if (e != cudaSuccess) rc = fail_cuda(h, "cudaEventCreate", e);
  for (int64_t it = 0; rc == SW_OK && it < nsteps; ++it) {
    pf.n = 0;
    int64_t nl = 0;
    e = h->fp32 ? enqueue_step<float>(h, h->stream, &pf, &nl) : enqueue_step<double>(h, h->stream, &pf, &nl);
    if (e == cudaSuccess) e = cudaStreamSynchronize(h->stream);
    if (e != cudaSuccess) {
      rc = fail_cuda(h, "sw_kernel_times step", e);
      break;
    }
    h->launches += nl;
    h->steps_total += 1;
    if (h->lm_open) h->done += 1;
    for (int i = 0; i < pf.n; ++i) {
      float t = 0.f;
      if ((e = cudaEventElapsedTime(&t, pf.ev[2 * i], pf.ev[2 * i + 1])) != cudaSuccess) {
        rc = fail_cuda(h, "cudaEventElapsedTime", e);
        break;
      }
      ms[pf.cls[i]] += t;
      launches[pf.cls[i]] += 1;
      bytes[pf.cls[i]] += pf.bytes[i];
    }
  }
  for (int i = 0; i < nev; ++i) cudaEventDestroy(pf.ev[i]);
  return rc;
}

extern "C" int sw_launch_count(sw_handle* h, int64_t* count) {
  if (!h || !count) return SW_EINVAL;
  *count = h->launches;
  return SW_OK;
}

extern "C" int sw_time(sw_handle* h, double* t) {
  if (!h || !t) return SW_EINVAL;
  *t = (double)h->steps_total * h->p.dt;
  return SW_OK;
}

extern "C" int sw_sync(sw_handle* h) {
  if (!h) return SW_EINVAL;
  CK(h, cudaStreamSynchronize(h->stream));
  return SW_OK;
}

extern "C" const char* sw_last_error(sw_handle* h) { return h ? h->err.c_str() : g_create_error.c_str(); }

extern "C" const char* sw_version(void) { return "lagmean-gb300 0.1"; }
