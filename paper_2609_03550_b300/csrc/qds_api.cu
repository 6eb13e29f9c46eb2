// qds_api.cu -- the C-ABI of the QDS field-step library (include/qds.h).
//
// The caller (PyTorch in the Python binding) owns all device memory of the
// field state and the sources; a handle owns only its descriptor tables, a
// step counter, a small diagnostics scratch and any captured CUDA graphs.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <map>
#include <string>
#include <tuple>
#include <vector>

#include "../../include/qds.h"
#include "qds_kernels.cuh"

using namespace qds;

namespace {

thread_local std::string g_err;

int fail(int code, const std::string &msg) {
  g_err = msg;
  return code;
}

#define CU(call)                                                                       \
  do {                                                                                 \
    cudaError_t e_ = (call);                                                           \
    if (e_ != cudaSuccess) return fail(QDS_ERR_CUDA, std::string(#call) + ": " + cudaGetErrorString(e_)); \
  } while (0)

constexpr int kThreads = 256;
// the step implementation behind QDS_STEP_DEFAULT
constexpr int kDefaultMode = QDS_STEP_FLAT;
constexpr size_t kAlign = 256;

size_t align_up(size_t x) { return (x + kAlign - 1) / kAlign * kAlign; }

bool is_fp32(const qds_params &p) { return (p.flags & QDS_FP32) != 0; }
bool is_scaled(const qds_params &p) { return (p.flags & (QDS_FP32 | QDS_SCALE_G)) != 0 && p.g != 0.0; }

// Stability and consistency rules (validated against the oracle's one-step
// map: the near-axis m/r terms need dr >= (m_max + 1/4) dx, the outer axion
// ghost needs dr >= 1.5 dx, and a mass widens both by (1 + dx m_a)).
int validate(const qds_params &p) {
  if (p.nx < 8 || p.nr < 4) return fail(QDS_ERR_INVALID_ARG, "nx must be >= 8 and nr >= 4");
  if ((double)15 * p.n_modes * p.nx * p.nr + (double)p.n_modes * p.nx > 2147483647.0)
    return fail(QDS_ERR_INVALID_ARG, "one instance must hold fewer than 2^31 state elements");
  if (p.n_modes < 1 || p.n_modes > 4) return fail(QDS_ERR_INVALID_ARG, "n_modes must be 1..4");
  if (p.modes)
    for (int k = 0; k < p.n_modes; k++)
      if (p.modes[k] != k) return fail(QDS_ERR_INVALID_ARG, "modes must be {0, 1, ..., n_modes-1}");
  if (!(p.dx > 0) || !(p.dr > 0) || !(p.dt > 0)) return fail(QDS_ERR_INVALID_ARG, "dx, dr, dt must be positive");
  if (std::fabs(p.dt - p.dx) > 1e-12 * p.dx) return fail(QDS_ERR_INVALID_ARG, "the QDS shift needs c*dt == dx (c = 1)");
  if (p.m_a < 0 || p.dx * p.m_a > 1.0) return fail(QDS_ERR_INVALID_ARG, "need 0 <= m_a and dx*m_a <= 1");
  double need = std::fmax(1.5, (p.n_modes - 1) + 0.25) * (1.0 + p.dx * p.m_a) * p.dx;
  if (p.dr < need * (1.0 - 1e-12)) {
    char b[160];
    std::snprintf(b, sizeof b, "unstable: dr = %g < %g (needs dr >= dx max(1.5, m_max+1/4)(1 + dx m_a))", p.dr, need);
    return fail(QDS_ERR_INVALID_ARG, b);
  }
  const uint32_t known = QDS_AXION | QDS_AREM | QDS_MOVING_WINDOW | QDS_X_PERIODIC | QDS_R_CLOSED | QDS_FP32 | QDS_SCALE_G;
  if (p.flags & ~known) return fail(QDS_ERR_INVALID_ARG, "unknown flag bits");
  if ((p.flags & QDS_MOVING_WINDOW) && (p.flags & QDS_X_PERIODIC))
    return fail(QDS_ERR_INVALID_ARG, "moving window and periodic x are exclusive");
  if ((p.flags & QDS_AREM) && !(p.flags & QDS_AXION)) return fail(QDS_ERR_INVALID_ARG, "QDS_AREM needs QDS_AXION");
  return QDS_OK;
}

size_t elem_bytes(const qds_params &p) { return is_fp32(p) ? 8 : 16; }

size_t half_bytes(const qds_params &p) { return align_up(state_elems(p.n_modes, p.nx, p.nr) * elem_bytes(p)); }

// two ping-pong copies of the state, then four scratch planes (Gamma_a and
// the three components of j_a) used by the pass-mode step
size_t instance_bytes(const qds_params &p) {
  return 2 * half_bytes(p) + align_up(4 * plane_elems(p.n_modes, p.nx, p.nr) * elem_bytes(p));
}

Geo pick_geo(const qds_params &p, int override_tx, int override_tr) {
  Geo g;
  g.TX = override_tx > 0 ? override_tx : 8;
  g.TR = override_tr > 0 ? override_tr : 32;
  if (override_tr <= 0) {
    size_t eb = elem_bytes(p);
    while (g.TR > 8 && (size_t)smem_layout(g, p.n_modes, p.flags).total * eb > 200 * 1024) g.TR /= 2;
  }
  return g;
}

}  // namespace

// Internal (not part of the C ABI): lets the other translation unit of the
// library report through qds_last_error().
__attribute__((visibility("hidden"))) void qds_internal_set_error(const std::string &m) { g_err = m; }

struct qds_handle {
  int n_inst = 0;
  std::vector<qds_params> params;
  std::vector<std::vector<int32_t>> modes;
  bool fp32 = false;
  uint32_t flags = 0;  // common flags (all instances share precision)
  char *state = nullptr;
  std::vector<size_t> inst_off;  // byte offset of each instance in the state arena
  // device tables
  void *d_inst = nullptr;  // Inst<R>[n_inst]
  Ctrl *d_ctrl = nullptr;
  double *d_partial = nullptr;
  double *d_diag = nullptr;
  int diag_blocks = 0;
  double *d_partial_all = nullptr;  // [n_inst][diag_all_blocks][4]
  double4 *d_scal = nullptr;        // per-instance diagnostic prefactors
  int diag_all_blocks = 0;
  // per-M launch groups
  struct Group {
    int M;
    Geo g;
    Smem L;
    int4 *d_tiles = nullptr;  // pass mode: interior tiles first, then edge tiles
    int ntiles = 0;
    int n_interior = 0;       // pass mode: tiles whose halo lies inside the window
    // warp-column passes P1 (31 output rows per warp) and P2 (30), interior first
    int4 *d_w[2] = {nullptr, nullptr};
    int nw[2] = {0, 0}, nw_interior[2] = {0, 0};
    // flat stage passes: (instance, first point, points, 0), interior first
    int4 *d_flat = nullptr;
    int nflat = 0, nflat_interior = 0;
    // the same per mode: (instance, first point, points, mode)
    int4 *d_flatk = nullptr;
    int nflatk = 0, nflatk_interior = 0;
    int q_base = 0;  // first of this group's work counters (interior, edge per stage)
  };
  // pass modes: the mode-count groups of a batch run on streams of their own
  // between a fork and a join event (independent instances)
  std::vector<cudaStream_t> gstream;
  std::vector<cudaEvent_t> gjoin;
  cudaEvent_t fork = nullptr;
  int *d_queue = nullptr;  // work counters of the persistent passes
  int n_queue = 0;
  int n_sm = 0;
  std::vector<Group> groups;
  std::vector<std::vector<char>> h_inst;  // host copy of the descriptors (per instance)
  int mode = QDS_STEP_DEFAULT;  // step implementation (qds_set_step_mode)
  // pass-mode tiles (one thread per point)
  std::vector<Group> pgroups;
  // graph cache: key (jx, jr, jt, sext, nsteps, stream)
  std::map<std::tuple<const void *, const void *, const void *, const void *, int, void *>, cudaGraphExec_t> graphs;
  const void *cur_src[4] = {nullptr, nullptr, nullptr, nullptr};
};

namespace {

template <class R>
void fill_inst(qds_handle *h, int i, const qds_params &p, void *base) {
  Inst<R> I;
  std::memset(&I, 0, sizeof I);
  I.nx = p.nx;
  I.nr = p.nr;
  I.M = p.n_modes;
  I.flags = p.flags;
  I.h = (R)p.dx;
  I.dr = (R)p.dr;
  I.inv_h = (R)(1.0 / p.dx);
  I.inv_dr = (R)(1.0 / p.dr);
  I.ma2 = (R)(p.m_a * p.m_a);
  const bool sc = is_scaled(p);
  I.gs = sc ? (R)1 : (R)p.g;
  I.gj = sc ? (R)1 : (R)p.g;
  size_t half = align_up(state_elems(p.n_modes, p.nx, p.nr) * sizeof(C<R>));
  I.state[0] = reinterpret_cast<C<R> *>((char *)base);
  I.state[1] = reinterpret_cast<C<R> *>((char *)base + half);
  I.scratch = reinterpret_cast<C<R> *>((char *)base + 2 * half);
  I.jx = I.jr = I.jt = I.sext = nullptr;
  h->h_inst[i].assign((char *)&I, (char *)&I + sizeof I);
}

template <class R>
void set_sources(qds_handle *h, const qds_sources *src) {
  for (int i = 0; i < h->n_inst; i++) {
    Inst<R> *I = reinterpret_cast<Inst<R> *>(h->h_inst[i].data());
    I->jx = src ? (const C<R> *)src->jx : nullptr;
    I->jr = src ? (const C<R> *)src->jr : nullptr;
    I->jt = src ? (const C<R> *)src->jth : nullptr;
    I->sext = src ? (const C<R> *)src->s_ext : nullptr;
  }
}

size_t inst_size(const qds_handle *h) { return h->fp32 ? sizeof(Inst<float>) : sizeof(Inst<double>); }

int upload_inst(qds_handle *h, cudaStream_t st) {
  const size_t sz = inst_size(h);
  std::vector<char> buf(sz * h->n_inst);
  for (int i = 0; i < h->n_inst; i++) std::memcpy(buf.data() + i * sz, h->h_inst[i].data(), sz);
  CU(cudaMemcpyAsync(h->d_inst, buf.data(), buf.size(), cudaMemcpyHostToDevice, st));
  CU(cudaStreamSynchronize(st));
  return QDS_OK;
}

template <class R, int M>
cudaError_t launch_group(qds_handle *h, const qds_handle::Group &G, cudaStream_t st) {
  const size_t smem = (size_t)G.L.total * sizeof(C<R>);
  step_kernel<R, M><<<G.ntiles, kThreads, smem, st>>>((const Inst<R> *)h->d_inst, G.d_tiles, h->d_ctrl, G.g, G.L);
  return cudaGetLastError();
}

template <class R, int M>
cudaError_t allow_smem(size_t bytes) {
  return cudaFuncSetAttribute(step_kernel<R, M>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
}

cudaError_t allow_smem_for(bool fp32, int M, size_t bytes) {
  if (fp32) {
    switch (M) { case 1: return allow_smem<float, 1>(bytes); case 2: return allow_smem<float, 2>(bytes);
                 case 3: return allow_smem<float, 3>(bytes); case 4: return allow_smem<float, 4>(bytes); }
  } else {
    switch (M) { case 1: return allow_smem<double, 1>(bytes); case 2: return allow_smem<double, 2>(bytes);
                 case 3: return allow_smem<double, 3>(bytes); case 4: return allow_smem<double, 4>(bytes); }
  }
  return cudaErrorInvalidValue;
}

template <class R, int M, int ST>
cudaError_t launch_pass(qds_handle *h, const qds_handle::Group &G, cudaStream_t st) {
  if (G.n_interior > 0)
    pass_kernel<R, M, ST, true><<<G.n_interior, kThreads, 0, st>>>((const Inst<R> *)h->d_inst, G.d_tiles, h->d_ctrl, G.g);
  if (G.ntiles > G.n_interior)
    pass_kernel<R, M, ST, false><<<G.ntiles - G.n_interior, kThreads, 0, st>>>(
        (const Inst<R> *)h->d_inst, G.d_tiles + G.n_interior, h->d_ctrl, G.g);
  return cudaGetLastError();
}

template <class R, int M, int ST>
cudaError_t launch_flat(qds_handle *h, const qds_handle::Group &G, cudaStream_t st) {
  if (G.nflat_interior > 0)
    flat_pass_kernel<R, M, ST, true><<<G.nflat_interior, kThreads, 0, st>>>((const Inst<R> *)h->d_inst, G.d_flat,
                                                                            h->d_ctrl);
  if (G.nflat > G.nflat_interior)
    flat_pass_kernel<R, M, ST, false><<<G.nflat - G.nflat_interior, kThreads, 0, st>>>(
        (const Inst<R> *)h->d_inst, G.d_flat + G.nflat_interior, h->d_ctrl);
  return cudaGetLastError();
}

template <class R, int M, int ST, bool FAST>
int queue_grid(qds_handle *h, int nblocks) {
  int per_sm = 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, queue_pass_kernel<R, M, ST, FAST>, kThreads, 0) != cudaSuccess ||
      per_sm < 1)
    per_sm = 1;
  return std::max(1, std::min(nblocks, per_sm * h->n_sm));
}

template <class R, int M, int ST>
cudaError_t launch_queue(qds_handle *h, const qds_handle::Group &G, cudaStream_t st) {
  int *c = h->d_queue + G.q_base + 2 * ST;
  const int ni = G.nflat_interior, ne = G.nflat - G.nflat_interior;
  if (ni > 0)
    queue_pass_kernel<R, M, ST, true><<<queue_grid<R, M, ST, true>(h, ni), kThreads, 0, st>>>(
        (const Inst<R> *)h->d_inst, G.d_flat, ni, c, h->d_ctrl);
  if (ne > 0)
    queue_pass_kernel<R, M, ST, false><<<queue_grid<R, M, ST, false>(h, ne), kThreads, 0, st>>>(
        (const Inst<R> *)h->d_inst, G.d_flat + ni, ne, c + 1, h->d_ctrl);
  return cudaGetLastError();
}

template <class R, int M, int ST>
cudaError_t launch_flatk(qds_handle *h, const qds_handle::Group &G, cudaStream_t st) {
  if (G.nflatk_interior > 0)
    flatk_pass_kernel<R, M, ST, true><<<G.nflatk_interior, kThreads, 0, st>>>((const Inst<R> *)h->d_inst, G.d_flatk,
                                                                              h->d_ctrl);
  if (G.nflatk > G.nflatk_interior)
    flatk_pass_kernel<R, M, ST, false><<<G.nflatk - G.nflatk_interior, kThreads, 0, st>>>(
        (const Inst<R> *)h->d_inst, G.d_flatk + G.nflatk_interior, h->d_ctrl);
  return cudaGetLastError();
}

template <class R, int M, int PASS>
cudaError_t launch_warp_pass(qds_handle *h, const qds_handle::Group &G, cudaStream_t st) {
  const int q = PASS - 1;
  const size_t smem = warp_pass_smem<R, M>(PASS);
  if (G.nw_interior[q] > 0)
    warp_pass_kernel<R, M, PASS, true><<<G.nw_interior[q], kThreads, smem, st>>>((const Inst<R> *)h->d_inst, G.d_w[q],
                                                                              h->d_ctrl, G.g);
  if (G.nw[q] > G.nw_interior[q])
    warp_pass_kernel<R, M, PASS, false><<<G.nw[q] - G.nw_interior[q], kThreads, smem, st>>>(
        (const Inst<R> *)h->d_inst, G.d_w[q] + G.nw_interior[q], h->d_ctrl, G.g);
  return cudaGetLastError();
}

template <class R, int M>
cudaError_t allow_warp_smem_t() {
  cudaError_t e;
  if ((e = cudaFuncSetAttribute(warp_pass_kernel<R, M, 1, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)warp_pass_smem<R, M>(1))) != cudaSuccess) return e;
  if ((e = cudaFuncSetAttribute(warp_pass_kernel<R, M, 1, false>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)warp_pass_smem<R, M>(1))) != cudaSuccess) return e;
  if ((e = cudaFuncSetAttribute(warp_pass_kernel<R, M, 2, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)warp_pass_smem<R, M>(2))) != cudaSuccess) return e;
  return cudaFuncSetAttribute(warp_pass_kernel<R, M, 2, false>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)warp_pass_smem<R, M>(2));
}

cudaError_t allow_warp_smem(bool fp32, int M) {
  switch (M) {
    case 1: return fp32 ? allow_warp_smem_t<float, 1>() : allow_warp_smem_t<double, 1>();
    case 2: return fp32 ? allow_warp_smem_t<float, 2>() : allow_warp_smem_t<double, 2>();
    case 3: return fp32 ? allow_warp_smem_t<float, 3>() : allow_warp_smem_t<double, 3>();
    case 4: return fp32 ? allow_warp_smem_t<float, 4>() : allow_warp_smem_t<double, 4>();
  }
  return cudaErrorInvalidValue;
}

// One step of one mode-count group in pass mode: the two warp-column passes,
// the regenerated shift and (moving window) the zeroing of the rear column.
template <class R, int M>
cudaError_t launch_passes(qds_handle *h, const qds_handle::Group &G, uint32_t fl, int mode, cudaStream_t st) {
  const bool ax = (fl & (F_AXION | F_AREM)) != 0, ar = (fl & F_AREM) != 0, mw = (fl & F_MOVING_WINDOW) != 0;
  cudaError_t e;
  if (mode == QDS_STEP_FLAT_MODES) {
    if ((e = launch_flatk<R, M, ST_LEAP0>(h, G, st)) != cudaSuccess) return e;
    if (ax && (e = launch_flat<R, M, ST_SOURCE>(h, G, st)) != cudaSuccess) return e;
    if ((e = launch_flatk<R, M, ST_SHIFT0>(h, G, st)) != cudaSuccess) return e;
    if (ar && (e = launch_flat<R, M, ST_CURRENT>(h, G, st)) != cudaSuccess) return e;
    if (ar && (e = launch_flatk<R, M, ST_SHIFT1>(h, G, st)) != cudaSuccess) return e;
    if (mw && (e = launch_flatk<R, M, ST_ZERO>(h, G, st)) != cudaSuccess) return e;
    return cudaSuccess;
  }
  if (mode == QDS_STEP_QUEUE) {
    if ((e = launch_queue<R, M, ST_LEAP0>(h, G, st)) != cudaSuccess) return e;
    if (ax && (e = launch_queue<R, M, ST_SOURCE>(h, G, st)) != cudaSuccess) return e;
    if ((e = launch_queue<R, M, ST_SHIFT0>(h, G, st)) != cudaSuccess) return e;
    if (ar && (e = launch_queue<R, M, ST_CURRENT>(h, G, st)) != cudaSuccess) return e;
    if (ar && (e = launch_queue<R, M, ST_SHIFT1>(h, G, st)) != cudaSuccess) return e;
    if (mw && (e = launch_queue<R, M, ST_ZERO>(h, G, st)) != cudaSuccess) return e;
    return cudaSuccess;
  }
  if (mode == QDS_STEP_FLAT) {
    if ((e = launch_flat<R, M, ST_LEAP0>(h, G, st)) != cudaSuccess) return e;
    if (ax && (e = launch_flat<R, M, ST_SOURCE>(h, G, st)) != cudaSuccess) return e;
    if ((e = launch_flat<R, M, ST_SHIFT0>(h, G, st)) != cudaSuccess) return e;
    if (ar && (e = launch_flat<R, M, ST_CURRENT>(h, G, st)) != cudaSuccess) return e;
    if (ar && (e = launch_flat<R, M, ST_SHIFT1>(h, G, st)) != cudaSuccess) return e;
    if (mw && (e = launch_flat<R, M, ST_ZERO>(h, G, st)) != cudaSuccess) return e;
    return cudaSuccess;
  }
  if (mode == QDS_STEP_STAGES) {
    if ((e = launch_pass<R, M, ST_LEAP0>(h, G, st)) != cudaSuccess) return e;
    if (ax && (e = launch_pass<R, M, ST_SOURCE>(h, G, st)) != cudaSuccess) return e;
  } else if ((e = launch_warp_pass<R, M, 1>(h, G, st)) != cudaSuccess) {
    return e;
  }
  if (mode == QDS_STEP_WARP) {
    if ((e = launch_warp_pass<R, M, 2>(h, G, st)) != cudaSuccess) return e;
  } else {
    // phi is formed in ST_SHIFT0 and the regenerated leapfrog in ST_CURRENT
    if ((e = launch_pass<R, M, ST_SHIFT0>(h, G, st)) != cudaSuccess) return e;
    if (ar && (e = launch_pass<R, M, ST_CURRENT>(h, G, st)) != cudaSuccess) return e;
  }
  if (ar && (e = launch_pass<R, M, ST_SHIFT1>(h, G, st)) != cudaSuccess) return e;
  if (mw && (e = launch_pass<R, M, ST_ZERO>(h, G, st)) != cudaSuccess) return e;
  return cudaSuccess;
}

template <class R>
cudaError_t launch_step(qds_handle *h, cudaStream_t st) {
  const int mode = h->mode == QDS_STEP_DEFAULT ? kDefaultMode : h->mode;
  if (mode != QDS_STEP_FUSED) {
    if (mode == QDS_STEP_QUEUE) zero_counters_kernel<<<1, 256, 0, st>>>(h->d_queue, h->n_queue);
    const bool fork = h->pgroups.size() > 1;
    cudaError_t e = cudaSuccess;
    if (fork && (e = cudaEventRecord(h->fork, st)) != cudaSuccess) return e;
    for (size_t gi = 0; gi < h->pgroups.size(); gi++) {
      const auto &G = h->pgroups[gi];
      cudaStream_t gs = st;
      if (fork) {
        gs = h->gstream[gi];
        if ((e = cudaStreamWaitEvent(gs, h->fork, 0)) != cudaSuccess) return e;
      }
      uint32_t fl = 0;
      for (int i = 0; i < h->n_inst; i++)
        if (h->params[i].n_modes == G.M) fl |= h->params[i].flags;
      switch (G.M) {
        case 1: e = launch_passes<R, 1>(h, G, fl, mode, gs); break;
        case 2: e = launch_passes<R, 2>(h, G, fl, mode, gs); break;
        case 3: e = launch_passes<R, 3>(h, G, fl, mode, gs); break;
        case 4: e = launch_passes<R, 4>(h, G, fl, mode, gs); break;
        default: e = cudaErrorInvalidValue;
      }
      if (e != cudaSuccess) return e;
      if (fork) {
        if ((e = cudaEventRecord(h->gjoin[gi], gs)) != cudaSuccess) return e;
        if ((e = cudaStreamWaitEvent(st, h->gjoin[gi], 0)) != cudaSuccess) return e;
      }
    }
    advance_kernel<<<1, 32, 0, st>>>(h->d_ctrl, 1);
    return cudaGetLastError();
  }
  for (const auto &G : h->groups) {
    cudaError_t e = cudaSuccess;
    switch (G.M) {
      case 1: e = launch_group<R, 1>(h, G, st); break;
      case 2: e = launch_group<R, 2>(h, G, st); break;
      case 3: e = launch_group<R, 3>(h, G, st); break;
      case 4: e = launch_group<R, 4>(h, G, st); break;
      default: e = cudaErrorInvalidValue;
    }
    if (e != cudaSuccess) return e;
  }
  advance_kernel<<<1, 32, 0, st>>>(h->d_ctrl, 1);
  return cudaGetLastError();
}

cudaError_t launch_steps(qds_handle *h, int n, cudaStream_t st) {
  for (int k = 0; k < n; k++) {
    cudaError_t e = h->fp32 ? launch_step<float>(h, st) : launch_step<double>(h, st);
    if (e != cudaSuccess) return e;
  }
  return cudaSuccess;
}

int build(qds_handle *h, int n, const qds_params *params, void *state, size_t bytes, int tx, int tr) {
  if (n < 1) return fail(QDS_ERR_INVALID_ARG, "need at least one instance");
  const bool fp32 = is_fp32(params[0]);
  size_t need = 0;
  for (int i = 0; i < n; i++) {
    int rc = validate(params[i]);
    if (rc) return rc;
    if (is_fp32(params[i]) != fp32) return fail(QDS_ERR_INVALID_ARG, "all instances of a batch share one precision");
    need += instance_bytes(params[i]);
  }
  if (!state) return fail(QDS_ERR_INVALID_ARG, "state buffer is NULL");
  if (reinterpret_cast<uintptr_t>(state) % kAlign) return fail(QDS_ERR_INVALID_ARG, "state buffer must be 256-byte aligned");
  if (bytes < need) return fail(QDS_ERR_INVALID_ARG, "state buffer too small (see qds_state_bytes)");
  h->n_inst = n;
  h->fp32 = fp32;
  h->state = (char *)state;
  h->params.assign(params, params + n);
  h->modes.resize(n);
  h->h_inst.resize(n);
  h->flags = params[0].flags;
  size_t off = 0;
  for (int i = 0; i < n; i++) {
    h->inst_off.push_back(off);
    if (fp32) fill_inst<float>(h, i, params[i], h->state + off);
    else fill_inst<double>(h, i, params[i], h->state + off);
    off += instance_bytes(params[i]);
  }
  CU(cudaMalloc(&h->d_inst, inst_size(h) * n));
  CU(cudaMalloc(&h->d_ctrl, sizeof(Ctrl)));
  CU(cudaMemset(h->d_ctrl, 0, sizeof(Ctrl)));
  h->diag_blocks = 592;
  CU(cudaMalloc(&h->d_partial, sizeof(double) * 4 * h->diag_blocks));
  CU(cudaMalloc(&h->d_diag, sizeof(double) * 4));
  h->diag_all_blocks = n >= 64 ? 8 : 64;
  CU(cudaMalloc(&h->d_partial_all, sizeof(double) * 4 * h->diag_all_blocks * n));
  {
    std::vector<double4> sc(n);
    for (int i = 0; i < n; i++) {
      const bool s_ = is_scaled(params[i]);
      const double g2 = s_ ? params[i].g * params[i].g : 1.0;
      sc[i] = make_double4(3.14159265358979323846 * params[i].dr * params[i].dx, g2, g2 * g2, g2);
    }
    CU(cudaMalloc(&h->d_scal, sizeof(double4) * n));
    CU(cudaMemcpy(h->d_scal, sc.data(), sizeof(double4) * n, cudaMemcpyHostToDevice));
  }
  // tiles grouped by mode count
  for (int M = 1; M <= 4; M++) {
    std::vector<int4> tl;
    Geo g{};
    Smem L{};
    uint32_t fl_union = 0;
    bool any = false;
    for (int i = 0; i < n; i++)
      if (params[i].n_modes == M) { fl_union |= params[i].flags; any = true; }
    if (!any) continue;
    qds_params pg = params[0];
    pg.n_modes = M;
    pg.flags = fl_union;
    g = pick_geo(pg, tx, tr);
    L = smem_layout(g, M, fl_union);
    for (int i = 0; i < n; i++) {
      if (params[i].n_modes != M) continue;
      for (int x0 = 0; x0 < params[i].nx; x0 += g.TX)
        for (int r0 = 0; r0 < params[i].nr; r0 += g.TR) tl.push_back(make_int4(i, x0, r0, 0));
    }
    qds_handle::Group G;
    G.M = M;
    G.g = g;
    G.L = L;
    G.ntiles = (int)tl.size();
    CU(cudaMalloc(&G.d_tiles, sizeof(int4) * tl.size()));
    CU(cudaMemcpy(G.d_tiles, tl.data(), sizeof(int4) * tl.size(), cudaMemcpyHostToDevice));
    const size_t smem = (size_t)L.total * elem_bytes(pg);
    if (smem > 227 * 1024) return fail(QDS_ERR_UNSUPPORTED, "tile does not fit in shared memory");
    CU(allow_smem_for(fp32, M, smem));
    h->groups.push_back(G);
    // pass mode: 8 x 32 points per CTA, one point per thread
    {
      qds_handle::Group P;
      P.M = M;
      P.g.TX = kThreads / 32;
      P.g.TR = 32;
      P.L = Smem{};
      std::vector<int4> pt, edge;
      for (int i = 0; i < n; i++) {
        if (params[i].n_modes != M) continue;
        const bool per = (params[i].flags & QDS_X_PERIODIC) != 0;
        for (int x0 = 0; x0 < params[i].nx; x0 += P.g.TX)
          for (int r0 = 0; r0 < params[i].nr; r0 += P.g.TR) {
            // interior: columns x0-2 .. x0+TX+1 are cells and x0+TX is a real face
            const bool inner = per ? (params[i].nx >= P.g.TX + 4) : (x0 >= 2 && x0 + P.g.TX + 2 <= params[i].nx - 1);
            (inner ? pt : edge).push_back(make_int4(i, x0, r0, 0));
          }
      }
      P.n_interior = (int)pt.size();
      pt.insert(pt.end(), edge.begin(), edge.end());
      P.ntiles = (int)pt.size();
      CU(cudaMalloc(&P.d_tiles, sizeof(int4) * pt.size()));
      CU(cudaMemcpy(P.d_tiles, pt.data(), sizeof(int4) * pt.size(), cudaMemcpyHostToDevice));
      // warp-column passes: (instance, x0, row of lane 0, first output row)
      for (int q = 0; q < 2; q++) {
        const int stride = q == 0 ? 31 : 30;
        std::vector<int4> wi, we;
        for (int i = 0; i < n; i++) {
          if (params[i].n_modes != M) continue;
          const bool per = (params[i].flags & QDS_X_PERIODIC) != 0;
          for (int x0 = 0; x0 < params[i].nx; x0 += P.g.TX)
            for (int r0 = 0; r0 < params[i].nr; r0 += stride) {
              const bool inner = per ? (params[i].nx >= P.g.TX + 4) : (x0 >= 2 && x0 + P.g.TX + 2 <= params[i].nx - 1);
              const int base = q == 0 ? r0 : (r0 > 0 ? r0 - 1 : 0);
              (inner ? wi : we).push_back(make_int4(i, x0, base, r0));
            }
        }
        P.nw_interior[q] = (int)wi.size();
        wi.insert(wi.end(), we.begin(), we.end());
        P.nw[q] = (int)wi.size();
        CU(cudaMalloc(&P.d_w[q], sizeof(int4) * wi.size()));
        CU(cudaMemcpy(P.d_w[q], wi.data(), sizeof(int4) * wi.size(), cudaMemcpyHostToDevice));
      }
      CU(allow_warp_smem(fp32, M));
      {
        std::vector<int4> fi, fe;
        for (int i = 0; i < n; i++) {
          if (params[i].n_modes != M) continue;
          const int nx_ = params[i].nx, nr_ = params[i].nr;
          const bool per = (params[i].flags & QDS_X_PERIODIC) != 0;
          const int total = nx_ * nr_;
          for (int q0 = 0; q0 < total; q0 += kThreads) {
            const int cnt = std::min(kThreads, total - q0);
            const int w0 = q0 / nr_, w1 = (q0 + cnt - 1) / nr_;
            // interior: columns w0-2 .. w1+2 are cells and w1+2 is a real face
            const bool inner = per ? (nx_ >= (w1 - w0 + 1) + 4) : (w0 >= 2 && w1 + 3 <= nx_ - 1);
            (inner ? fi : fe).push_back(make_int4(i, q0, cnt, 0));
          }
        }
        P.nflat_interior = (int)fi.size();
        fi.insert(fi.end(), fe.begin(), fe.end());
        P.nflat = (int)fi.size();
        CU(cudaMalloc(&P.d_flat, sizeof(int4) * fi.size()));
        CU(cudaMemcpy(P.d_flat, fi.data(), sizeof(int4) * fi.size(), cudaMemcpyHostToDevice));
        // per mode: every block of the point list once per mode
        std::vector<int4> ki, ke;
        for (int k = 0; k < M; k++)
          for (int b = 0; b < P.nflat; b++) {
            int4 v = fi[b];
            v.w = k;
            (b < P.nflat_interior ? ki : ke).push_back(v);
          }
        P.nflatk_interior = (int)ki.size();
        ki.insert(ki.end(), ke.begin(), ke.end());
        P.nflatk = (int)ki.size();
        CU(cudaMalloc(&P.d_flatk, sizeof(int4) * ki.size()));
        CU(cudaMemcpy(P.d_flatk, ki.data(), sizeof(int4) * ki.size(), cudaMemcpyHostToDevice));
      }
      P.q_base = 2 * (N_STAGE + 1) * (int)h->pgroups.size();  // stages 0 .. ST_ZERO
      h->pgroups.push_back(P);
    }
  }
  CU(cudaEventCreateWithFlags(&h->fork, cudaEventDisableTiming));
  for (size_t gi = 0; gi < h->pgroups.size(); gi++) {
    cudaStream_t gs;
    cudaEvent_t ev;
    CU(cudaStreamCreateWithFlags(&gs, cudaStreamNonBlocking));
    h->gstream.push_back(gs);
    CU(cudaEventCreateWithFlags(&ev, cudaEventDisableTiming));
    h->gjoin.push_back(ev);
  }
  h->n_queue = 2 * (N_STAGE + 1) * (int)h->pgroups.size();
  CU(cudaMalloc(&h->d_queue, sizeof(int) * std::max(1, h->n_queue)));
  CU(cudaMemset(h->d_queue, 0, sizeof(int) * std::max(1, h->n_queue)));
  {
    int dev = 0;
    CU(cudaGetDevice(&dev));
    CU(cudaDeviceGetAttribute(&h->n_sm, cudaDevAttrMultiProcessorCount, dev));
  }
  return upload_inst(h, 0);
}

void destroy(qds_handle *h) {
  if (!h) return;
  for (auto &kv : h->graphs) cudaGraphExecDestroy(kv.second);
  for (auto &G : h->groups) cudaFree(G.d_tiles);
  for (auto &G : h->pgroups) { cudaFree(G.d_tiles); cudaFree(G.d_w[0]); cudaFree(G.d_w[1]); cudaFree(G.d_flat); cudaFree(G.d_flatk); }
  cudaFree(h->d_queue);
  for (auto gs : h->gstream) cudaStreamDestroy(gs);
  for (auto ev : h->gjoin) cudaEventDestroy(ev);
  if (h->fork) cudaEventDestroy(h->fork);
  cudaFree(h->d_inst);
  cudaFree(h->d_ctrl);
  cudaFree(h->d_partial);
  cudaFree(h->d_diag);
  cudaFree(h->d_partial_all);
  cudaFree(h->d_scal);
  delete h;
}

}  // namespace

// ============================================================================
// Parameters of instance i, for the adjoint translation unit.
__attribute__((visibility("hidden"))) int qds_internal_params(const qds_handle *h, int i, qds_params *out) {
  if (!h) return fail(QDS_ERR_INVALID_ARG, "NULL handle");
  if (i < 0 || i >= h->n_inst) return fail(QDS_ERR_INVALID_ARG, "instance index out of range");
  *out = h->params[i];
  out->modes = nullptr;
  return QDS_OK;
}

extern "C" {

const char *qds_last_error(void) { return g_err.c_str(); }

size_t qds_state_bytes(const qds_params *p) {
  if (!p || validate(*p)) return 0;
  return instance_bytes(*p);
}

size_t qds_batch_state_bytes(int n, const qds_params *p) {
  if (n < 1 || !p) return 0;
  size_t s = 0;
  for (int i = 0; i < n; i++) {
    if (validate(p[i])) return 0;
    s += instance_bytes(p[i]);
  }
  return s;
}

int qds_create(const qds_params *p, void *state_dev, size_t bytes, qds_handle **out) {
  return qds_batch_create(1, p, state_dev, bytes, out);
}

int qds_batch_create(int n, const qds_params *p, void *state_dev, size_t bytes, qds_handle **out) {
  if (!out || !p) return fail(QDS_ERR_INVALID_ARG, "NULL argument");
  *out = nullptr;
  qds_handle *h = new qds_handle();
  int rc = build(h, n, p, state_dev, bytes, 0, 0);
  if (rc) { destroy(h); return rc; }
  *out = h;
  return QDS_OK;
}

int qds_set_tile(qds_handle *h, int tx, int tr) {
  if (!h) return fail(QDS_ERR_INVALID_ARG, "NULL handle");
  if (tx < 1 || tx > 64 || tr < 4 || tr > 128) return fail(QDS_ERR_INVALID_ARG, "tile out of range");
  std::vector<qds_params> ps = h->params;
  void *st = h->state;
  size_t bytes = qds_batch_state_bytes((int)ps.size(), ps.data());
  qds_handle *nh = new qds_handle();
  int rc = build(nh, (int)ps.size(), ps.data(), st, bytes, tx, tr);
  if (rc) { destroy(nh); return rc; }
  // keep the step counter
  CU(cudaMemcpy(nh->d_ctrl, h->d_ctrl, sizeof(Ctrl), cudaMemcpyDeviceToDevice));
  for (auto &kv : h->graphs) cudaGraphExecDestroy(kv.second);
  h->graphs.clear();
  for (auto &G : h->groups) cudaFree(G.d_tiles);
  cudaFree(h->d_inst); cudaFree(h->d_ctrl); cudaFree(h->d_partial); cudaFree(h->d_diag);
  cudaFree(h->d_partial_all); cudaFree(h->d_scal);
  for (auto &G : h->pgroups) { cudaFree(G.d_tiles); cudaFree(G.d_w[0]); cudaFree(G.d_w[1]); cudaFree(G.d_flat); cudaFree(G.d_flatk); }
  h->groups = nh->groups; h->pgroups = nh->pgroups; h->d_inst = nh->d_inst; h->d_ctrl = nh->d_ctrl;
  h->d_partial_all = nh->d_partial_all; h->d_scal = nh->d_scal;
  h->d_partial = nh->d_partial; h->d_diag = nh->d_diag; h->h_inst = nh->h_inst;
  cudaFree(h->d_queue);
  h->d_queue = nh->d_queue; h->n_queue = nh->n_queue; h->n_sm = nh->n_sm;
  nh->d_queue = nullptr;
  for (auto gs : h->gstream) cudaStreamDestroy(gs);
  for (auto ev : h->gjoin) cudaEventDestroy(ev);
  if (h->fork) cudaEventDestroy(h->fork);
  h->gstream = nh->gstream; h->gjoin = nh->gjoin; h->fork = nh->fork;
  nh->gstream.clear(); nh->gjoin.clear(); nh->fork = nullptr;
  nh->groups.clear(); nh->pgroups.clear(); nh->d_inst = nullptr; nh->d_ctrl = nullptr; nh->d_partial = nullptr;
  nh->d_diag = nullptr; nh->d_partial_all = nullptr; nh->d_scal = nullptr;
  delete nh;
  return QDS_OK;
}

int qds_step_launches(const qds_handle *h) {
  if (!h) return 0;
  const int mode = h->mode == QDS_STEP_DEFAULT ? kDefaultMode : h->mode;
  if (mode == QDS_STEP_FUSED) return (int)h->groups.size() + 1;
  int n = mode == QDS_STEP_QUEUE ? 2 : 1;  // step counter (+ work counters)
  for (const auto &G : h->pgroups) {
    uint32_t fl = 0;
    for (int i = 0; i < h->n_inst; i++)
      if (h->params[i].n_modes == G.M) fl |= h->params[i].flags;
    const bool ax = (fl & (F_AXION | F_AREM)) != 0, ar = (fl & F_AREM) != 0, mw = (fl & F_MOVING_WINDOW) != 0;
    const int stage = (G.n_interior > 0) + (G.ntiles > G.n_interior);
    const int w1 = (G.nw_interior[0] > 0) + (G.nw[0] > G.nw_interior[0]);
    const int w2 = (G.nw_interior[1] > 0) + (G.nw[1] > G.nw_interior[1]);
    if (mode == QDS_STEP_FLAT || mode == QDS_STEP_FLAT_MODES || mode == QDS_STEP_QUEUE) {
      const int f = (G.nflat_interior > 0) + (G.nflat > G.nflat_interior);
      n += f * (2 + (ax ? 1 : 0) + (ar ? 2 : 0) + (mw ? 1 : 0));
      continue;
    }
    if (mode == QDS_STEP_STAGES) n += stage * (1 + (ax ? 1 : 0));
    else n += w1;
    if (mode == QDS_STEP_WARP) n += w2;
    else n += stage * (1 + (ar ? 1 : 0));
    n += stage * ((ar ? 1 : 0) + (mw ? 1 : 0));
  }
  return n;
}

int qds_set_fused(qds_handle *h, int fused) { return qds_set_step_mode(h, fused ? QDS_STEP_FUSED : QDS_STEP_DEFAULT); }

int qds_set_step_mode(qds_handle *h, int mode) {
  if (!h) return fail(QDS_ERR_INVALID_ARG, "NULL handle");
  if (mode < QDS_STEP_DEFAULT || mode > QDS_STEP_QUEUE) return fail(QDS_ERR_INVALID_ARG, "unknown step mode");
  h->mode = mode;
  for (auto &kv : h->graphs) cudaGraphExecDestroy(kv.second);
  h->graphs.clear();
  return QDS_OK;
}

int qds_get_tile(qds_handle *h, int *tx, int *tr, int *ntiles, int *smem_bytes) {
  if (!h || h->groups.empty()) return fail(QDS_ERR_INVALID_ARG, "NULL handle");
  const auto &G = h->groups[0];
  if (tx) *tx = G.g.TX;
  if (tr) *tr = G.g.TR;
  int nt = 0;
  for (const auto &g : h->groups) nt += g.ntiles;
  if (ntiles) *ntiles = nt;
  if (smem_bytes) *smem_bytes = G.L.total * (h->fp32 ? 8 : 16);
  return QDS_OK;
}

void qds_free(qds_handle *h) { destroy(h); }

int qds_set_state_i(qds_handle *h, int i, const void *src, void *stream) {
  if (!h || !src || i < 0 || i >= h->n_inst) return fail(QDS_ERR_INVALID_ARG, "bad handle, instance or source");
  cudaStream_t st = (cudaStream_t)stream;
  const qds_params &p = h->params[i];
  const double g = p.g;
  const bool sc = is_scaled(p);
  const double s_ax = sc ? 1.0 / g : 1.0, s_ar = sc ? 1.0 / (g * g) : 1.0;
  const size_t half = half_bytes(p);
  char *b = h->state + h->inst_off[i];
  if (h->fp32)
    import_kernel<float><<<592, kThreads, 0, st>>>((const double2 *)src, (C<float> *)b, (C<float> *)(b + half),
                                                   p.n_modes, p.nx, p.nr, s_ax, s_ar);
  else
    import_kernel<double><<<592, kThreads, 0, st>>>((const double2 *)src, (C<double> *)b, (C<double> *)(b + half),
                                                    p.n_modes, p.nx, p.nr, s_ax, s_ar);
  CU(cudaGetLastError());
  reset_kernel<<<1, 32, 0, st>>>(h->d_ctrl);
  CU(cudaGetLastError());
  return QDS_OK;
}

int qds_set_state(qds_handle *h, const void *src, void *stream) { return qds_set_state_i(h, 0, src, stream); }

int qds_get_state_i(qds_handle *h, int i, void *dst, void *stream) {
  if (!h || !dst || i < 0 || i >= h->n_inst) return fail(QDS_ERR_INVALID_ARG, "bad handle, instance or destination");
  cudaStream_t st = (cudaStream_t)stream;
  const qds_params &p = h->params[i];
  const bool sc = is_scaled(p);
  const double s_ax = sc ? p.g : 1.0, s_ar = sc ? p.g * p.g : 1.0;
  const size_t half = half_bytes(p);
  char *b = h->state + h->inst_off[i];
  if (h->fp32)
    export_kernel<float><<<592, kThreads, 0, st>>>((const C<float> *)b, (const C<float> *)(b + half), h->d_ctrl,
                                                   (double2 *)dst, p.n_modes, p.nx, p.nr, p.flags, s_ax, s_ar);
  else
    export_kernel<double><<<592, kThreads, 0, st>>>((const C<double> *)b, (const C<double> *)(b + half), h->d_ctrl,
                                                    (double2 *)dst, p.n_modes, p.nx, p.nr, p.flags, s_ax, s_ar);
  CU(cudaGetLastError());
  return QDS_OK;
}

int qds_get_state(qds_handle *h, void *dst, void *stream) { return qds_get_state_i(h, 0, dst, stream); }

int qds_step(qds_handle *h, const qds_sources *src, int nsteps, void *stream) {
  if (!h) return fail(QDS_ERR_INVALID_ARG, "NULL handle");
  if (nsteps < 0) return fail(QDS_ERR_INVALID_ARG, "nsteps < 0");
  if (nsteps == 0) return QDS_OK;
  if (src && h->n_inst != 1 && (src->jx || src->jr || src->jth || src->s_ext))
    return fail(QDS_ERR_UNSUPPORTED, "sources are per instance; batched handles take none");
  cudaStream_t st = (cudaStream_t)stream;
  const void *s4[4] = {src ? src->jx : nullptr, src ? src->jr : nullptr, src ? src->jth : nullptr,
                       src ? src->s_ext : nullptr};
  if (std::memcmp(s4, h->cur_src, sizeof s4) != 0) {
    if (h->fp32) set_sources<float>(h, src);
    else set_sources<double>(h, src);
    int rc = upload_inst(h, st);
    if (rc) return rc;
    std::memcpy(h->cur_src, s4, sizeof s4);
  }
  // Multi-step calls replay a captured graph of G launches.
  const int G = 16;
  if (nsteps < G) {
    cudaError_t e = launch_steps(h, nsteps, st);
    if (e != cudaSuccess) return fail(QDS_ERR_CUDA, std::string("step launch: ") + cudaGetErrorString(e));
    return QDS_OK;
  }
  auto key = std::make_tuple(s4[0], s4[1], s4[2], s4[3], G, (void *)st);
  auto it = h->graphs.find(key);
  if (it == h->graphs.end()) {
    cudaStream_t cs;
    CU(cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking));
    cudaGraph_t graph;
    CU(cudaStreamBeginCapture(cs, cudaStreamCaptureModeThreadLocal));
    cudaError_t e = launch_steps(h, G, cs);
    cudaError_t e2 = cudaStreamEndCapture(cs, &graph);
    cudaStreamDestroy(cs);
    if (e != cudaSuccess || e2 != cudaSuccess)
      return fail(QDS_ERR_CUDA, std::string("graph capture: ") + cudaGetErrorString(e != cudaSuccess ? e : e2));
    cudaGraphExec_t exec;
    CU(cudaGraphInstantiate(&exec, graph, 0));
    cudaGraphDestroy(graph);
    it = h->graphs.emplace(key, exec).first;
  }
  int full = nsteps / G, rem = nsteps % G;
  for (int k = 0; k < full; k++) CU(cudaGraphLaunch(it->second, st));
  if (rem) {
    cudaError_t e = launch_steps(h, rem, st);
    if (e != cudaSuccess) return fail(QDS_ERR_CUDA, std::string("step launch: ") + cudaGetErrorString(e));
  }
  return QDS_OK;
}

int qds_diagnostics_i(qds_handle *h, int i, double *out_host, double *profile_dev, void *stream) {
  if (!h || !out_host || i < 0 || i >= h->n_inst) return fail(QDS_ERR_INVALID_ARG, "bad handle, instance or output");
  cudaStream_t st = (cudaStream_t)stream;
  const qds_params &p = h->params[i];
  const bool sc = is_scaled(p);
  const double g2 = sc ? p.g * p.g : 1.0;
  const size_t half = half_bytes(p);
  char *b = h->state + h->inst_off[i];
  const double pref = 3.14159265358979323846 * p.dr * p.dx;
  if (h->fp32)
    diag_partial_kernel<float><<<h->diag_blocks, kThreads, 0, st>>>((const C<float> *)b, (const C<float> *)(b + half),
                                                                    h->d_ctrl, p.n_modes, p.nx, p.nr, p.dr, p.m_a * p.m_a, h->d_partial);
  else
    diag_partial_kernel<double><<<h->diag_blocks, kThreads, 0, st>>>((const C<double> *)b, (const C<double> *)(b + half),
                                                                     h->d_ctrl, p.n_modes, p.nx, p.nr, p.dr, p.m_a * p.m_a, h->d_partial);
  CU(cudaGetLastError());
  diag_final_kernel<<<1, 32, 0, st>>>(h->d_partial, h->diag_blocks, pref, g2, g2 * g2, g2, h->d_diag);
  CU(cudaGetLastError());
  if (profile_dev) {
    if (h->fp32)
      profile_kernel<float><<<p.nx, kThreads, 0, st>>>((const C<float> *)b, (const C<float> *)(b + half), h->d_ctrl,
                                                       p.n_modes, p.nx, p.nr, p.dr, p.flags, profile_dev);
    else
      profile_kernel<double><<<p.nx, kThreads, 0, st>>>((const C<double> *)b, (const C<double> *)(b + half), h->d_ctrl,
                                                        p.n_modes, p.nx, p.nr, p.dr, p.flags, profile_dev);
    CU(cudaGetLastError());
  }
  CU(cudaMemcpyAsync(out_host, h->d_diag, sizeof(double) * 4, cudaMemcpyDeviceToHost, st));
  CU(cudaStreamSynchronize(st));
  return QDS_OK;
}

int qds_diagnostics(qds_handle *h, double *out_host, double *profile_dev, void *stream) {
  return qds_diagnostics_i(h, 0, out_host, profile_dev, stream);
}

int qds_num_instances(const qds_handle *h) { return h ? h->n_inst : 0; }

int qds_diagnostics_all(qds_handle *h, double *out_dev, void *stream) {
  if (!h || !out_dev) return fail(QDS_ERR_INVALID_ARG, "bad handle or output");
  cudaStream_t st = (cudaStream_t)stream;
  dim3 grid(h->diag_all_blocks, h->n_inst);
  if (h->fp32)
    diag_partial_all_kernel<float><<<grid, kThreads, 0, st>>>((const Inst<float> *)h->d_inst, h->d_ctrl, h->d_partial_all);
  else
    diag_partial_all_kernel<double><<<grid, kThreads, 0, st>>>((const Inst<double> *)h->d_inst, h->d_ctrl, h->d_partial_all);
  CU(cudaGetLastError());
  diag_final_all_kernel<<<(h->n_inst + 127) / 128, 128, 0, st>>>(h->d_partial_all, h->diag_all_blocks, h->d_scal,
                                                                  h->n_inst, out_dev);
  CU(cudaGetLastError());
  return QDS_OK;
}

}  // extern "C"
