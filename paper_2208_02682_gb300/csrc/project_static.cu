// project_static.cu -- sw_project_static: projection of one physical field
// onto the 2/3-dealiased spectral box with no device allocation.
//
// Same kernels as the initial-condition and output transforms of a handle
// (FP64 row forward pass, column forward pass with the 2/3 mask, column
// inverse pass, row inverse pass); the mixed and spectral intermediates and
// the twiddle table live in the file-scope array below instead of memory
// obtained from cudaMalloc.
#include <cuda_runtime.h>

#include <mutex>
#include <string>

#include "../../include/lagmean.h"
#include "launch.cuh"

using namespace lm;

namespace lm {
cudaError_t prepare_kernels_f64();
void set_handleless_error(const std::string& msg);
}  // namespace lm

// Scratch shared by every call on a device; each GPU that loads the library
// holds it until the process exits.
static __device__ __align__(256) unsigned char g_project_scratch[SW_PROJECT_STATIC_BYTES];

// The pass-ordered FP64 twiddle table of the N-point transforms (entry
// r*Ns + k - 1 of the pass with stride Ns and radix R: exp(-2 pi i r k/(Ns R))).
__global__ void k_static_twiddles(double2* tw, int N, int log2N) {
  const int t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t < N - 1) {
    // the pass whose index range [Ns - 1, Ns R - 1) holds t
    int lNs = 0, lr = fft_pass_lr(log2N, 0);
    for (int p = 1; p < fft_num_passes(log2N) && t + 1 >= (1 << (lNs + lr)); ++p) {
      lNs += lr;
      lr = fft_pass_lr(log2N, p);
    }
    const int r = (t + 1) >> lNs, k = (t + 1) & ((1 << lNs) - 1);
    double s, c;
    sincospi(2.0 * (double)(r * k) / (double)(1 << (lNs + lr)), &s, &c);
    tw[t] = make_double2(c, -s);
  }
}

namespace {
std::mutex g_mu;
const int kMaxDevices = 256;
void* g_scratch_addr[kMaxDevices] = {};

size_t a256(size_t x) { return (x + 255) & ~(size_t)255; }

// Device address of the scratch array for the current device, resolved once
// per device (host code cannot use the symbol itself as a device pointer).
int scratch_for_device(void** out) {
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) {
    set_handleless_error(std::string("sw_project_static: cudaGetDevice: ") + cudaGetErrorString(e));
    return SW_ECUDA;
  }
  if (dev < 0 || dev >= kMaxDevices) {
    set_handleless_error("sw_project_static: device ordinal out of range");
    return SW_EINVAL;
  }
  std::lock_guard<std::mutex> lock(g_mu);
  if (!g_scratch_addr[dev]) {
    void* p = nullptr;
    e = cudaGetSymbolAddress(&p, g_project_scratch);
    if (e != cudaSuccess || !p) {
      set_handleless_error(std::string("sw_project_static: cudaGetSymbolAddress: ") + cudaGetErrorString(e));
      return SW_ECUDA;
    }
    e = prepare_kernels_f64();
    if (e != cudaSuccess) {
      set_handleless_error(std::string("sw_project_static: kernel set-up: ") + cudaGetErrorString(e));
      return SW_ECUDA;
    }
    g_scratch_addr[dev] = p;
  }
  *out = g_scratch_addr[dev];
  return SW_OK;
}
}  // namespace

extern "C" int sw_project_static(const double* in, double* out, int N, void* stream) {
  if (!in || !out) {
    set_handleless_error("sw_project_static: in and out must be device pointers");
    return SW_EINVAL;
  }
  if (N < 16 || N > SW_PROJECT_STATIC_MAX_N || (N & (N - 1)) != 0) {
    set_handleless_error("sw_project_static: N must be a power of two in [16, " +
                         std::to_string(SW_PROJECT_STATIC_MAX_N) + "]");
    return SW_EINVAL;
  }
  Geom g;
  g.N = N;
  g.log2N = 0;
  while ((1 << g.log2N) < N) ++g.log2N;
  g.K = (N - 1) / 3;
  g.KX = g.K + 1;
  g.KXP = (g.KX + 3) / 4 * 4;
  g.NY = 2 * g.K + 1;
  g.ms = (long long)g.NY * g.KXP;
  g.mi = (long long)g.N * g.KXP;
  g.np = (long long)g.N * g.N;
  const size_t o_spec = a256((size_t)g.mi * sizeof(double2));
  const size_t o_tw = o_spec + a256((size_t)g.ms * sizeof(double2));
  const size_t need = o_tw + a256((size_t)N * sizeof(double2));
  if (need > (size_t)SW_PROJECT_STATIC_BYTES) {
    set_handleless_error("sw_project_static: scratch of " + std::to_string(need) + " bytes exceeds the " +
                         std::to_string(SW_PROJECT_STATIC_BYTES) + "-byte static array");
    return SW_EINVAL;
  }
  void* base = nullptr;
  int rc = scratch_for_device(&base);
  if (rc != SW_OK) return rc;
  double2* mixed = (double2*)base;
  double2* spec = (double2*)((char*)base + o_spec);
  double2* tw = (double2*)((char*)base + o_tw);
  cudaStream_t s = (cudaStream_t)stream;

  k_static_twiddles<<<(N + 255) / 256, 256, 0, s>>>(tw, N, g.log2N);
  cudaError_t e = cudaGetLastError();
  const int B = row_block_rows(N);
  if (e == cudaSuccess) {
    RowFwdArgs<double> rf = {};
    rf.src = in;
    rf.dst = mixed;
    rf.tw = tw;
    rf.g = g;
    rf.B = B;
    rf.npairs = 1;
    rf.a_idx[0] = 0;
    rf.b_idx[0] = -1;
    rf.oa[0] = 0;
    rf.ob[0] = -1;
    e = launch_row_fwd<double>(rf, s);
  }
  if (e == cudaSuccess) {
    ColFwdArgs<double> cf;
    cf.src = mixed;
    cf.dst = spec;
    cf.tw = tw;
    cf.g = g;
    cf.nout = 1;
    cf.src_idx[0] = cf.dst_idx[0] = 0;
    e = launch_col_fwd<double>(cf, s);
  }
  if (e == cudaSuccess) {
    ColInvArgs<double> ci;
    ci.src = spec;
    ci.dst = mixed;
    ci.tw = tw;
    ci.g = g;
    ci.nout = 1;
    ci.src_idx[0] = 0;
    ci.src2_idx[0] = -1;
    ci.op[0] = OP_ID;
    ci.dst_idx[0] = 0;
    e = launch_col_inv<double>(ci, s);
  }
  if (e == cudaSuccess) {
    RowInvArgs<double, double> ri = {};
    ri.src = mixed;
    ri.dst = out;
    ri.dst_stride = g.np;
    ri.tw = tw;
    ri.g = g;
    ri.B = B;
    ri.npairs = 1;
    ri.a_idx[0] = 0;
    ri.b_idx[0] = -1;
    ri.oa[0] = 0;
    ri.ob[0] = -1;
    ri.sa[0] = 1.0;
    e = launch_row_inv<double, double>(ri, s);
  }
  if (e != cudaSuccess) {
    set_handleless_error(std::string("sw_project_static: launch: ") + cudaGetErrorString(e));
    return SW_ECUDA;
  }
  return SW_OK;
}
