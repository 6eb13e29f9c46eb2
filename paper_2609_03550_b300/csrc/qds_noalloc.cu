// qds_noalloc.cu -- qds_advance_noalloc(): the pass-mode field step for
// callers that cannot allocate device memory.
//
// Some callers cannot call cudaMalloc: code running inside a host callback
// or a memory-pool-managed runtime that forbids allocations after start-up,
// plug-ins that must not grow the device footprint of a host application,
// or real-time loops where an allocation may stall or fail.  The regular
// path (qds_create) allocates small descriptor tables and instantiates CUDA
// graphs.  This entry point allocates nothing: its descriptor, step counter,
// block table and the four scratch planes of the pass-mode step (Gamma_a and
// the three components of j_a) live in one file-scope device array of
// QDS_NOALLOC_SCRATCH_BYTES bytes, which every GPU that loads the library
// holds until the process exits.  The caller provides the inputs, the
// outputs and the working state.
#include <cuda.h>
#include <cuda_runtime.h>
#include <cudaTypedefs.h>

#include <algorithm>
#include <cstring>
#include <mutex>
#include <string>
#include <vector>

#include "../../include/qds.h"
#include "qds_kernels.cuh"

using namespace qds;

namespace {

static __device__ __align__(256) unsigned char g_noalloc_scratch[QDS_NOALLOC_SCRATCH_BYTES];

}  // namespace

// defined in qds_api.cu: sets the message that qds_last_error() returns
void qds_internal_set_error(const std::string &m);

namespace {

int fail_na(int code, const std::string &m) {
  qds_internal_set_error(m);
  return code;
}

// Device address of the scratch array, looked up with the device current
// the first time a call runs in a CUDA context of that device (again after
// the context was replaced, e.g. by cudaDeviceReset, which invalidates the
// old address).  The host-side name g_noalloc_scratch is only a stand-in.
constexpr int kMaxDevices = 64;
std::mutex g_mu;
void *g_addr[kMaxDevices] = {nullptr};
unsigned long long g_ctx_id[kMaxDevices] = {0};

// Unique id of the current CUDA context (0 if it cannot be read).
unsigned long long current_context_id() {
  static PFN_cuCtxGetCurrent_v4000 get_cur = nullptr;
  static PFN_cuCtxGetId_v12000 get_id = nullptr;
  static std::once_flag once;
  std::call_once(once, [] {
    void *p = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuCtxGetCurrent", &p, 4000, cudaEnableDefault, &q) == cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      get_cur = reinterpret_cast<PFN_cuCtxGetCurrent_v4000>(p);
    if (cudaGetDriverEntryPointByVersion("cuCtxGetId", &p, 12000, cudaEnableDefault, &q) == cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      get_id = reinterpret_cast<PFN_cuCtxGetId_v12000>(p);
  });
  CUcontext ctx = nullptr;
  unsigned long long id = 0;
  if (!get_cur || !get_id || get_cur(&ctx) != CUDA_SUCCESS || !ctx || get_id(ctx, &id) != CUDA_SUCCESS) return 0;
  return id;
}

int scratch_address(void **out) {
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return fail_na(QDS_ERR_CUDA, std::string("cudaGetDevice: ") + cudaGetErrorString(e));
  if (dev < 0 || dev >= kMaxDevices) return fail_na(QDS_ERR_UNSUPPORTED, "device index out of range");
  std::lock_guard<std::mutex> lk(g_mu);
  // cudaFree(0) makes the runtime bind this thread to the device's context
  // (created on first use), so that its id can be read
  if ((e = cudaFree(nullptr)) != cudaSuccess) return fail_na(QDS_ERR_CUDA, std::string("cudaFree(0): ") + cudaGetErrorString(e));
  const unsigned long long id = current_context_id();
  if (!g_addr[dev] || id == 0 || id != g_ctx_id[dev]) {
    void *p = nullptr;
    e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
    if (e != cudaSuccess || !p)
      return fail_na(QDS_ERR_CUDA, std::string("cudaGetSymbolAddress: ") + cudaGetErrorString(e));
    g_addr[dev] = p;
    g_ctx_id[dev] = id;
  }
  *out = g_addr[dev];
  return QDS_OK;
}

constexpr int kThr = 256;
size_t up256(size_t x) { return (x + 255) / 256 * 256; }

template <class R, int M>
cudaError_t run_steps(const Inst<R> *d_inst, const int4 *d_blocks, int nblocks, Ctrl *d_ctrl, uint32_t fl,
                      int nsteps, cudaStream_t st) {
  const bool ax = (fl & (F_AXION | F_AREM)) != 0, ar = (fl & F_AREM) != 0, mw = (fl & F_MOVING_WINDOW) != 0;
  for (int n = 0; n < nsteps; n++) {
    flat_pass_kernel<R, M, ST_LEAP0, false><<<nblocks, kThr, 0, st>>>(d_inst, d_blocks, d_ctrl);
    if (ax) flat_pass_kernel<R, M, ST_SOURCE, false><<<nblocks, kThr, 0, st>>>(d_inst, d_blocks, d_ctrl);
    flat_pass_kernel<R, M, ST_SHIFT0, false><<<nblocks, kThr, 0, st>>>(d_inst, d_blocks, d_ctrl);
    if (ar) flat_pass_kernel<R, M, ST_CURRENT, false><<<nblocks, kThr, 0, st>>>(d_inst, d_blocks, d_ctrl);
    if (ar) flat_pass_kernel<R, M, ST_SHIFT1, false><<<nblocks, kThr, 0, st>>>(d_inst, d_blocks, d_ctrl);
    if (mw) flat_pass_kernel<R, M, ST_ZERO, false><<<nblocks, kThr, 0, st>>>(d_inst, d_blocks, d_ctrl);
    advance_kernel<<<1, 32, 0, st>>>(d_ctrl, 1);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
  }
  return cudaSuccess;
}

template <class R>
int advance(const qds_params &p, const void *in, void *out, void *work, size_t work_bytes, int nsteps,
            cudaStream_t st) {
  const int M = p.n_modes, nx = p.nx, nr = p.nr, ld = row_stride<R>(nr);
  const size_t P = plane_elems(M, nx, ld);
  const size_t half = up256(state_elems(M, nx, ld) * sizeof(C<R>));
  if (work_bytes < 2 * half) return fail_na(QDS_ERR_INVALID_ARG, "work buffer smaller than two state copies");
  if (reinterpret_cast<uintptr_t>(work) % 256) return fail_na(QDS_ERR_INVALID_ARG, "work buffer must be 256-byte aligned");
  // blocks of 256 consecutive points (x, r order), every one checked
  std::vector<int4> tiles;
  for (int q0 = 0; q0 < nx * nr; q0 += kThr) tiles.push_back(make_int4(0, q0, std::min(kThr, nx * nr - q0), 0));
  const size_t off_ctrl = up256(sizeof(Inst<R>));
  const size_t off_tiles = off_ctrl + up256(sizeof(Ctrl));
  const size_t off_scr = off_tiles + up256(tiles.size() * sizeof(int4));
  const size_t need = off_scr + 4 * P * sizeof(C<R>);
  if (need > (size_t)QDS_NOALLOC_SCRATCH_BYTES)
    return fail_na(QDS_ERR_INVALID_ARG, "grid too large for the no-allocation scratch (" + std::to_string(need) +
                                            " > " + std::to_string((size_t)QDS_NOALLOC_SCRATCH_BYTES) + " bytes)");
  void *base = nullptr;
  int rc = scratch_address(&base);
  if (rc) return rc;
  char *b = static_cast<char *>(base);
  Inst<R> I;
  std::memset(&I, 0, sizeof I);
  I.nx = nx;
  I.nr = nr;
  I.ld = ld;
  I.M = M;
  I.flags = p.flags;
  I.h = (R)p.dx;
  I.dr = (R)p.dr;
  I.inv_h = (R)(1.0 / p.dx);
  I.inv_dr = (R)(1.0 / p.dr);
  I.ma2 = (R)(p.m_a * p.m_a);
  const bool sc = (p.flags & (QDS_FP32 | QDS_SCALE_G)) != 0 && p.g != 0.0;
  I.gs = sc ? (R)1 : (R)p.g;
  I.gj = sc ? (R)1 : (R)p.g;
  I.state[0] = reinterpret_cast<C<R> *>(work);
  I.state[1] = reinterpret_cast<C<R> *>(static_cast<char *>(work) + half);
  I.scratch = reinterpret_cast<C<R> *>(b + off_scr);
  Ctrl c;
  std::memset(&c, 0, sizeof c);
  cudaError_t e;
  // the calls share the array: descriptor, counter and tiles are rewritten,
  // and the scratch planes cleared, at the start of every call
  if ((e = cudaMemcpyAsync(b, &I, sizeof I, cudaMemcpyHostToDevice, st)) != cudaSuccess ||
      (e = cudaMemcpyAsync(b + off_ctrl, &c, sizeof c, cudaMemcpyHostToDevice, st)) != cudaSuccess ||
      (e = cudaMemcpyAsync(b + off_tiles, tiles.data(), tiles.size() * sizeof(int4), cudaMemcpyHostToDevice, st)) != cudaSuccess ||
      (e = cudaMemsetAsync(b + off_scr, 0, 4 * P * sizeof(C<R>), st)) != cudaSuccess ||
      (e = cudaStreamSynchronize(st)) != cudaSuccess)
    return fail_na(QDS_ERR_CUDA, std::string("scratch set-up: ") + cudaGetErrorString(e));
  const double s_ax = sc ? 1.0 / p.g : 1.0, s_ar = sc ? 1.0 / (p.g * p.g) : 1.0;
  import_kernel<R><<<592, kThr, 0, st>>>((const double2 *)in, I.state[0], I.state[1], M, nx, nr, ld, s_ax, s_ar);
  const Inst<R> *d_inst = reinterpret_cast<const Inst<R> *>(b);
  const int4 *d_tiles = reinterpret_cast<const int4 *>(b + off_tiles);
  Ctrl *d_ctrl = reinterpret_cast<Ctrl *>(b + off_ctrl);
  switch (M) {
    case 1: e = run_steps<R, 1>(d_inst, d_tiles, (int)tiles.size(), d_ctrl, p.flags, nsteps, st); break;
    case 2: e = run_steps<R, 2>(d_inst, d_tiles, (int)tiles.size(), d_ctrl, p.flags, nsteps, st); break;
    case 3: e = run_steps<R, 3>(d_inst, d_tiles, (int)tiles.size(), d_ctrl, p.flags, nsteps, st); break;
    case 4: e = run_steps<R, 4>(d_inst, d_tiles, (int)tiles.size(), d_ctrl, p.flags, nsteps, st); break;
    default: e = cudaErrorInvalidValue;
  }
  if (e != cudaSuccess) return fail_na(QDS_ERR_CUDA, std::string("step launch: ") + cudaGetErrorString(e));
  const double g_ax = sc ? p.g : 1.0, g_ar = sc ? p.g * p.g : 1.0;
  export_kernel<R><<<592, kThr, 0, st>>>(I.state[0], I.state[1], d_ctrl, (double2 *)out, M, nx, nr, ld, p.flags, g_ax, g_ar);
  if ((e = cudaGetLastError()) != cudaSuccess) return fail_na(QDS_ERR_CUDA, std::string("export: ") + cudaGetErrorString(e));
  return QDS_OK;
}

}  // namespace

extern "C" int qds_advance_noalloc(const qds_params *p, const void *state_in_dev, void *state_out_dev,
                                   void *work_dev, size_t work_bytes, int nsteps, void *stream) {
  if (!p || !state_in_dev || !state_out_dev || !work_dev || nsteps < 0)
    return fail_na(QDS_ERR_INVALID_ARG, "NULL argument or negative step count");
  if (qds_state_bytes(p) == 0) return QDS_ERR_INVALID_ARG;  // qds_last_error() names the rule
  cudaStream_t st = (cudaStream_t)stream;
  if (p->flags & QDS_FP32) return advance<float>(*p, state_in_dev, state_out_dev, work_dev, work_bytes, nsteps, st);
  return advance<double>(*p, state_in_dev, state_out_dev, work_dev, work_bytes, nsteps, st);
}
