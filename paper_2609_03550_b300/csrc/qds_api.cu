// qds_api.cu -- the C-ABI of the QDS field-step library (include/qds.h).
//
// The caller (PyTorch in the Python binding) owns all device memory of the
// field state and the sources; a handle owns only its descriptor tables, the
// tensor maps of the bulk copies, a step counter, a small diagnostics
// scratch and any captured CUDA graphs.
#include <cuda.h>
#include <cuda_runtime.h>
#include <cudaTypedefs.h>

#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <map>
#include <mutex>
#include <string>
#include <tuple>
#include <vector>

#include "../../include/qds.h"
#include "qds_march.cuh"

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
constexpr size_t kAlign = 256;

size_t align_up(size_t x) { return (x + kAlign - 1) / kAlign * kAlign; }

bool is_fp32(const qds_params &p) { return (p.flags & QDS_FP32) != 0; }
bool is_scaled(const qds_params &p) { return (p.flags & (QDS_FP32 | QDS_SCALE_G)) != 0 && p.g != 0.0; }

// Stability and consistency rules (validated against the oracle's one-step
// map: the near-axis m/r terms need dr >= (m_max + 1/4) dx, the outer axion
// ghost needs dr >= 1.5 dx, and a mass widens both by (1 + dx m_a)).
int validate(const qds_params &p) {
  if (p.nx < 8 || p.nr < 4) return fail(QDS_ERR_INVALID_ARG, "nx must be >= 8 and nr >= 4");
  if (p.nx > (1 << 24) || p.nr > 32768) return fail(QDS_ERR_INVALID_ARG, "nx must be <= 2^24 and nr <= 32768");
  const double ld = (p.flags & QDS_FP32) ? p.nr + (p.nr & 1) : p.nr;  // row stride of the working layout
  if ((double)15 * p.n_modes * p.nx * ld + (double)p.n_modes * p.nx > 2147483647.0)
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
int row_ld(const qds_params &p) { return is_fp32(p) ? row_stride<float>(p.nr) : row_stride<double>(p.nr); }

size_t half_bytes(const qds_params &p) { return align_up(state_elems(p.n_modes, p.nx, row_ld(p)) * elem_bytes(p)); }

// two ping-pong copies of the state, then four scratch planes (Gamma_a and
// the three components of j_a)
size_t instance_bytes(const qds_params &p) {
  return 2 * half_bytes(p) + align_up(4 * plane_elems(p.n_modes, p.nx, row_ld(p)) * elem_bytes(p));
}

// ---------------------------------------------------------------------------
// x-marching launch plan
// ---------------------------------------------------------------------------
// Ring rows per CTA the kernels are compiled for: 32 and 64 in FP32, 32 in
// FP64 (a warp is then 32 rows of one mode).  A request is rounded down to
// one of these; 0 gives the default, 64 in FP32.
int march_rows(bool fp32, int req) {
  if (!fp32) return 32;
  return req == 0 || req >= 64 ? 64 : 32;
}

PFN_cuTensorMapEncodeTiled_v12000 encode_fn() {
  static std::once_flag once;
  static PFN_cuTensorMapEncodeTiled_v12000 fn = nullptr;
  std::call_once(once, [] {
    void *p = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) == cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      fn = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(p);
  });
  return fn;
}

// Tensor map over planes [nplanes][M][nx][ld] of complex elements at base:
// dims (row, column, mode, plane), box (RB rows, one column, all modes,
// box_planes planes).  8-byte integer elements: one per FP32 complex, two
// per FP64 complex.  Coordinates outside the tensor read as zero.
int encode_map(CUtensorMap *out, void *base, bool fp32, int M, int nx, int nr, int ld, int nplanes, int RB,
               int box_planes) {
  auto fn = encode_fn();
  if (!fn) return fail(QDS_ERR_CUDA, "cuTensorMapEncodeTiled is not available from the driver");
  const cuuint64_t w = fp32 ? 1 : 2;  // 8-byte words per complex
  cuuint64_t dims[4] = {w * (cuuint64_t)nr, (cuuint64_t)nx, (cuuint64_t)M, (cuuint64_t)nplanes};
  const cuuint64_t eb = 8 * w;
  cuuint64_t strides[3] = {eb * ld, eb * ld * nx, eb * ld * nx * M};
  cuuint32_t box[4] = {(cuuint32_t)(w * RB), 1, (cuuint32_t)M, (cuuint32_t)box_planes};
  cuuint32_t es[4] = {1, 1, 1, 1};
  CUresult r = fn(out, CU_TENSOR_MAP_DATA_TYPE_INT64, 4, base, dims, strides, box, es, CU_TENSOR_MAP_INTERLEAVE_NONE,
                  CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  if (r != CUDA_SUCCESS) {
    char b[200];
    std::snprintf(b, sizeof b, "cuTensorMapEncodeTiled failed (%d) for nx=%d nr=%d M=%d rows=%d", (int)r, nx, nr, M, RB);
    return fail(QDS_ERR_CUDA, b);
  }
  return QDS_OK;
}

// Work items of one kernel kind for one instance: bands of rows (see
// march_bands) times segments of columns.
void march_items(std::vector<MarchItem> &out, int inst, int nx, int nr, int RB, int halo, int seg) {
  march_bands(nr, RB, halo, [&](int r0, int r1, int rb0) {
    for (int xa = 0; xa < nx; xa += seg) {
      MarchItem it{};
      it.inst = inst; it.r0 = r0; it.r1 = r1; it.rb0 = rb0; it.xa = xa; it.xb = std::min(nx, xa + seg);
      out.push_back(it);
    }
  });
}

}  // namespace

// Internal (not part of the C ABI): lets the other translation units of the
// library report through qds_last_error().
__attribute__((visibility("hidden"))) void qds_internal_set_error(const std::string &m) { g_err = m; }

struct qds_handle {
  int n_inst = 0;
  std::vector<qds_params> params;
  bool fp32 = false;
  char *state = nullptr;
  std::vector<size_t> inst_off;  // byte offset of each instance in the state arena
  // device tables
  void *d_inst = nullptr;  // Inst<R>[n_inst]
  Ctrl *d_ctrl = nullptr;
  double *d_partial = nullptr;
  double *d_diag = nullptr;
  int diag_blocks = 0;
  double *d_partial_all = nullptr;  // [n_inst][diag_all_blocks][4]
  Scal4 *d_scal = nullptr;        // per-instance diagnostic prefactors
  int diag_all_blocks = 0;
  MarchMaps *d_maps = nullptr;      // per instance
  // per mode count
  struct Group {
    int M = 0;
    uint32_t flags = 0;  // union of the flags of its instances
    // flat stage passes: (instance, first point, points, 0), interior first
    int4 *d_flat = nullptr;
    int nflat = 0, nflat_interior = 0;
    // x-marching: K1 and K2 work items and shared-memory plans
    MarchItem *d_items[2] = {nullptr, nullptr};
    int nitems[2] = {0, 0};
    int rows[2] = {0, 0};
    MarchGeo geo[2];
  };
  std::vector<Group> groups;
  // the mode-count groups of a batch run on streams of their own between a
  // fork and a join event (independent instances)
  std::vector<cudaStream_t> gstream;
  std::vector<cudaEvent_t> gjoin;
  cudaEvent_t fork = nullptr;
  std::vector<std::vector<char>> h_inst;  // host copy of the descriptors (per instance)
  int mode = QDS_STEP_DEFAULT;  // step implementation (qds_set_step_mode)
  unsigned long long host_step = 0;  // mirror of the device step counter (steps since the last state import)
  int seg = 0;                  // march: columns per CTA (0: default)
  int rows_override = 0;        // march: rows per CTA (0: default)
  // graph cache: key (steps per graph, stream); the kernels read the source
  // pointers from the device descriptors at run time
  std::map<std::tuple<int, void *>, cudaGraphExec_t> graphs;
};

namespace {

constexpr int kDefaultMode = QDS_STEP_FLAT;  // measured faster on the batched scan
constexpr int kDefaultSeg = 128;

template <class R>
void fill_inst(qds_handle *h, int i, const qds_params &p, void *base) {
  Inst<R> I;
  std::memset(&I, 0, sizeof I);
  I.nx = p.nx;
  I.nr = p.nr;
  I.ld = row_ld(p);
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
  size_t half = half_bytes(p);
  I.state[0] = reinterpret_cast<C<R> *>((char *)base);
  I.state[1] = reinterpret_cast<C<R> *>((char *)base + half);
  I.scratch = reinterpret_cast<C<R> *>((char *)base + 2 * half);
  I.jx = I.jr = I.jt = I.sext = nullptr;
  h->h_inst[i].assign((char *)&I, (char *)&I + sizeof I);
}

// Sources of instance i (NULL clears), stride elements apart from step to
// step of a qds_step call (0: the same arrays every step).
template <class R>
void set_sources_i(qds_handle *h, int i, const qds_sources *src, long long stride) {
  Inst<R> *I = reinterpret_cast<Inst<R> *>(h->h_inst[i].data());
  I->jx = src ? (const C<R> *)src->jx : nullptr;
  I->jr = src ? (const C<R> *)src->jr : nullptr;
  I->jt = src ? (const C<R> *)src->jth : nullptr;
  I->sext = src ? (const C<R> *)src->s_ext : nullptr;
  I->sstride = stride;
}

bool sources_equal(const qds_handle *h, int i, const qds_sources *src, long long stride) {
  const void *s4[4] = {src ? src->jx : nullptr, src ? src->jr : nullptr, src ? src->jth : nullptr,
                       src ? src->s_ext : nullptr};
  if (h->fp32) {
    const Inst<float> *I = reinterpret_cast<const Inst<float> *>(h->h_inst[i].data());
    return I->jx == s4[0] && I->jr == s4[1] && I->jt == s4[2] && I->sext == s4[3] && I->sstride == stride;
  }
  const Inst<double> *I = reinterpret_cast<const Inst<double> *>(h->h_inst[i].data());
  return I->jx == s4[0] && I->jr == s4[1] && I->jt == s4[2] && I->sext == s4[3] && I->sstride == stride;
}

bool any_strided(const qds_handle *h) {
  for (int i = 0; i < h->n_inst; i++) {
    long long s, si;
    if (h->fp32) {
      const Inst<float> *I = reinterpret_cast<const Inst<float> *>(h->h_inst[i].data());
      s = I->sstride; si = I->istride;
    } else {
      const Inst<double> *I = reinterpret_cast<const Inst<double> *>(h->h_inst[i].data());
      s = I->sstride; si = I->istride;
    }
    if (s || si) return true;
  }
  return false;
}

// Injection arrays of instance i (NULL: none).
template <class R>
void set_inflow_i(qds_handle *h, int i, const void *tr_plus, const void *tth_minus, long long stride) {
  Inst<R> *I = reinterpret_cast<Inst<R> *>(h->h_inst[i].data());
  I->in_rp = (const C<R> *)tr_plus;
  I->in_tm = (const C<R> *)tth_minus;
  I->istride = stride;
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

template <class R, int M, int RB, int KIND>
cudaError_t launch_march_rb(qds_handle *h, const qds_handle::Group &G, cudaStream_t st) {
  march_kernel<R, M, RB, KIND><<<G.nitems[KIND], march_threads<M, RB, KIND>(), G.geo[KIND].bytes, st>>>(
      (const Inst<R> *)h->d_inst, h->d_maps, G.d_items[KIND], h->d_ctrl);
  return cudaGetLastError();
}

template <class R, int M, int KIND>
cudaError_t launch_march(qds_handle *h, const qds_handle::Group &G, cudaStream_t st) {
  if constexpr (sizeof(R) == 4) {
    if (G.rows[KIND] == 64) return launch_march_rb<R, M, 64, KIND>(h, G, st);
  }
  return launch_march_rb<R, M, 32, KIND>(h, G, st);
}

template <class R, int M, int RB>
cudaError_t allow_march_smem_rb() {
  const int b0 = march_geo<R>(0, M, RB).bytes, b1 = march_geo<R>(1, M, RB).bytes;
  cudaError_t e = cudaFuncSetAttribute(march_kernel<R, M, RB, 0>, cudaFuncAttributeMaxDynamicSharedMemorySize, b0);
  if (e != cudaSuccess) return e;
  return cudaFuncSetAttribute(march_kernel<R, M, RB, 1>, cudaFuncAttributeMaxDynamicSharedMemorySize, b1);
}

template <int M>
cudaError_t allow_march_smem_m(bool fp32) {
  if (!fp32) return allow_march_smem_rb<double, M, 32>();
  cudaError_t e = allow_march_smem_rb<float, M, 32>();
  if (e != cudaSuccess) return e;
  return allow_march_smem_rb<float, M, 64>();
}

cudaError_t allow_march_smem(bool fp32, int M) {
  switch (M) {
    case 1: return allow_march_smem_m<1>(fp32);
    case 2: return allow_march_smem_m<2>(fp32);
    case 3: return allow_march_smem_m<3>(fp32);
    case 4: return allow_march_smem_m<4>(fp32);
  }
  return cudaErrorInvalidValue;
}

// One step of one mode-count group: the flat stage passes (six launches
// over interior and edge blocks) or the two x-marching kernels.
template <class R, int M>
cudaError_t launch_group(qds_handle *h, const qds_handle::Group &G, int mode, cudaStream_t st) {
  const uint32_t fl = G.flags;
  const bool ax = (fl & (F_AXION | F_AREM)) != 0, ar = (fl & F_AREM) != 0, mw = (fl & F_MOVING_WINDOW) != 0;
  cudaError_t e;
  if (mode == QDS_STEP_MARCH) {
    if ((e = launch_march<R, M, 0>(h, G, st)) != cudaSuccess) return e;
    if (ar && (e = launch_march<R, M, 1>(h, G, st)) != cudaSuccess) return e;
    return cudaSuccess;
  }
  if ((e = launch_flat<R, M, ST_LEAP0>(h, G, st)) != cudaSuccess) return e;
  if (ax && (e = launch_flat<R, M, ST_SOURCE>(h, G, st)) != cudaSuccess) return e;
  if ((e = launch_flat<R, M, ST_SHIFT0>(h, G, st)) != cudaSuccess) return e;
  if (ar && (e = launch_flat<R, M, ST_CURRENT>(h, G, st)) != cudaSuccess) return e;
  if (ar && (e = launch_flat<R, M, ST_SHIFT1>(h, G, st)) != cudaSuccess) return e;
  if (mw && (e = launch_flat<R, M, ST_ZERO>(h, G, st)) != cudaSuccess) return e;
  return cudaSuccess;
}

int effective_mode(const qds_handle *h) { return h->mode == QDS_STEP_DEFAULT ? kDefaultMode : h->mode; }

template <class R>
cudaError_t launch_step(qds_handle *h, cudaStream_t st) {
  const int mode = effective_mode(h);
  const bool fork = h->groups.size() > 1;
  cudaError_t e = cudaSuccess;
  if (fork && (e = cudaEventRecord(h->fork, st)) != cudaSuccess) return e;
  for (size_t gi = 0; gi < h->groups.size(); gi++) {
    const auto &G = h->groups[gi];
    cudaStream_t gs = st;
    if (fork) {
      gs = h->gstream[gi];
      if ((e = cudaStreamWaitEvent(gs, h->fork, 0)) != cudaSuccess) return e;
    }
    switch (G.M) {
      case 1: e = launch_group<R, 1>(h, G, mode, gs); break;
      case 2: e = launch_group<R, 2>(h, G, mode, gs); break;
      case 3: e = launch_group<R, 3>(h, G, mode, gs); break;
      case 4: e = launch_group<R, 4>(h, G, mode, gs); break;
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

cudaError_t launch_steps(qds_handle *h, int n, cudaStream_t st) {
  for (int k = 0; k < n; k++) {
    cudaError_t e = h->fp32 ? launch_step<float>(h, st) : launch_step<double>(h, st);
    if (e != cudaSuccess) return e;
  }
  return cudaSuccess;
}

void drop_graphs(qds_handle *h) {
  for (auto &kv : h->graphs) cudaGraphExecDestroy(kv.second);
  h->graphs.clear();
}

// (Re)build the x-marching work items and tensor maps of every group.
int build_march(qds_handle *h) {
  for (auto &G : h->groups) {
    for (int kind = 0; kind < 2; kind++) {
      cudaFree(G.d_items[kind]);
      G.d_items[kind] = nullptr;
      const int RB = march_rows(h->fp32, h->rows_override);
      const int halo = kind == 0 ? kHalo1 : kHalo2;
      G.rows[kind] = RB;
      G.geo[kind] = h->fp32 ? march_geo<float>(kind, G.M, RB) : march_geo<double>(kind, G.M, RB);
      if (G.geo[kind].bytes > 227 * 1024) return fail(QDS_ERR_UNSUPPORTED, "march tile does not fit in shared memory");
      std::vector<MarchItem> items;
      const int seg = h->seg > 0 ? h->seg : kDefaultSeg;
      for (int i = 0; i < h->n_inst; i++)
        if (h->params[i].n_modes == G.M) march_items(items, i, h->params[i].nx, h->params[i].nr, RB, halo, seg);
      G.nitems[kind] = (int)items.size();
      CU(cudaMalloc(&G.d_items[kind], sizeof(MarchItem) * std::max<size_t>(1, items.size())));
      CU(cudaMemcpy(G.d_items[kind], items.data(), sizeof(MarchItem) * items.size(), cudaMemcpyHostToDevice));
    }
    CU(allow_march_smem(h->fp32, G.M));
  }
  // tensor maps of every instance (box rows of its group)
  std::vector<MarchMaps> maps(h->n_inst);
  std::memset(maps.data(), 0, sizeof(MarchMaps) * maps.size());
  for (int i = 0; i < h->n_inst; i++) {
    const qds_params &p = h->params[i];
    const qds_handle::Group *G = nullptr;
    for (auto &g : h->groups)
      if (g.M == p.n_modes) G = &g;
    const int ld = row_ld(p);
    char *base = h->state + h->inst_off[i];
    const size_t half = half_bytes(p);
    for (int par = 0; par < 2; par++) {
      int rc = encode_map(&maps[i].k1[par], base + par * half, h->fp32, p.n_modes, p.nx, p.nr, ld, NFIELD, G->rows[0], 9);
      if (rc) return rc;
      rc = encode_map(&maps[i].k2[par], base + par * half, h->fp32, p.n_modes, p.nx, p.nr, ld, NFIELD, G->rows[1], 6);
      if (rc) return rc;
    }
    int rc = encode_map(&maps[i].ja, base + 2 * half, h->fp32, p.n_modes, p.nx, p.nr, ld, 4, G->rows[1], 3);
    if (rc) return rc;
  }
  if (!h->d_maps) CU(cudaMalloc(&h->d_maps, sizeof(MarchMaps) * h->n_inst));
  CU(cudaMemcpy(h->d_maps, maps.data(), sizeof(MarchMaps) * h->n_inst, cudaMemcpyHostToDevice));
  return QDS_OK;
}

int build(qds_handle *h, int n, const qds_params *params, void *state, size_t bytes) {
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
  for (auto &p : h->params) p.modes = nullptr;
  h->h_inst.resize(n);
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
    std::vector<Scal4> sc(n);
    for (int i = 0; i < n; i++) {
      const bool s_ = is_scaled(params[i]);
      const double g2 = s_ ? params[i].g * params[i].g : 1.0;
      sc[i] = Scal4{3.14159265358979323846 * params[i].dr * params[i].dx, g2, g2 * g2, g2};
    }
    CU(cudaMalloc(&h->d_scal, sizeof(Scal4) * n));
    CU(cudaMemcpy(h->d_scal, sc.data(), sizeof(Scal4) * n, cudaMemcpyHostToDevice));
  }
  for (int M = 1; M <= 4; M++) {
    qds_handle::Group G;
    G.M = M;
    bool any = false;
    for (int i = 0; i < n; i++)
      if (params[i].n_modes == M) { G.flags |= params[i].flags; any = true; }
    if (!any) continue;
    // flat passes: blocks of 256 consecutive points of one instance
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
    G.nflat_interior = (int)fi.size();
    fi.insert(fi.end(), fe.begin(), fe.end());
    G.nflat = (int)fi.size();
    CU(cudaMalloc(&G.d_flat, sizeof(int4) * fi.size()));
    CU(cudaMemcpy(G.d_flat, fi.data(), sizeof(int4) * fi.size(), cudaMemcpyHostToDevice));
    h->groups.push_back(G);
  }
  int rc = build_march(h);
  if (rc) return rc;
  CU(cudaEventCreateWithFlags(&h->fork, cudaEventDisableTiming));
  for (size_t gi = 0; gi < h->groups.size(); gi++) {
    cudaStream_t gs;
    cudaEvent_t ev;
    CU(cudaStreamCreateWithFlags(&gs, cudaStreamNonBlocking));
    h->gstream.push_back(gs);
    CU(cudaEventCreateWithFlags(&ev, cudaEventDisableTiming));
    h->gjoin.push_back(ev);
  }
  return upload_inst(h, 0);
}

void destroy(qds_handle *h) {
  if (!h) return;
  drop_graphs(h);
  for (auto &G : h->groups) {
    cudaFree(G.d_flat);
    cudaFree(G.d_items[0]);
    cudaFree(G.d_items[1]);
  }
  for (auto gs : h->gstream) cudaStreamDestroy(gs);
  for (auto ev : h->gjoin) cudaEventDestroy(ev);
  if (h->fork) cudaEventDestroy(h->fork);
  cudaFree(h->d_inst);
  cudaFree(h->d_ctrl);
  cudaFree(h->d_partial);
  cudaFree(h->d_diag);
  cudaFree(h->d_partial_all);
  cudaFree(h->d_scal);
  cudaFree(h->d_maps);
  delete h;
}

// Device error bits -> status (synchronises the stream).
int read_status(qds_handle *h, cudaStream_t st) {
  Ctrl c;
  CU(cudaMemcpyAsync(&c, h->d_ctrl, sizeof c, cudaMemcpyDeviceToHost, st));
  CU(cudaStreamSynchronize(st));
  if (c.err & kErrTimeout) return fail(QDS_ERR_TIMEOUT, "a bulk copy of the step kernel did not complete in time");
  if (c.err & kErrNonfinite) return fail(QDS_ERR_NONFINITE, "non-finite field values (NaN or Inf) in the state");
  return QDS_OK;
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

// Row stride of instance i's working layout, for the adjoint translation unit.
__attribute__((visibility("hidden"))) int qds_internal_layout(const qds_handle *h, int i, int *ld) {
  if (!h || i < 0 || i >= h->n_inst) return fail(QDS_ERR_INVALID_ARG, "bad handle or instance");
  *ld = row_ld(h->params[i]);
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
  int rc = build(h, n, p, state_dev, bytes);
  if (rc) { destroy(h); return rc; }
  *out = h;
  return QDS_OK;
}

int qds_set_tile(qds_handle *h, int rows, int cols) {
  if (!h) return fail(QDS_ERR_INVALID_ARG, "NULL handle");
  if (rows < 0 || rows > 256 || cols < 0 || cols > (1 << 20) || (cols > 0 && cols < 4))
    return fail(QDS_ERR_INVALID_ARG, "tile out of range (rows 0 or 24..256, columns 0 or >= 4)");
  const int old_rows = h->rows_override, old_seg = h->seg;
  h->rows_override = rows;
  h->seg = cols;
  int rc = build_march(h);
  if (rc) {
    h->rows_override = old_rows;
    h->seg = old_seg;
    const std::string msg = g_err;
    build_march(h);
    return fail(rc, msg);
  }
  drop_graphs(h);
  return QDS_OK;
}

int qds_get_tile(qds_handle *h, int *rows, int *cols, int *ntiles, int *smem_bytes) {
  if (!h || h->groups.empty()) return fail(QDS_ERR_INVALID_ARG, "NULL handle");
  const auto &G = h->groups[0];
  if (rows) *rows = G.rows[0];
  if (cols) *cols = h->seg > 0 ? h->seg : kDefaultSeg;
  int nt = 0;
  for (const auto &g : h->groups) nt += g.nitems[0] + g.nitems[1];
  if (ntiles) *ntiles = nt;
  if (smem_bytes) *smem_bytes = G.geo[0].bytes;
  return QDS_OK;
}

int qds_step_launches(const qds_handle *h) {
  if (!h) return 0;
  const int mode = effective_mode(h);
  int n = 1;  // step counter
  for (const auto &G : h->groups) {
    const bool ax = (G.flags & (F_AXION | F_AREM)) != 0, ar = (G.flags & F_AREM) != 0,
               mw = (G.flags & F_MOVING_WINDOW) != 0;
    if (mode == QDS_STEP_MARCH) {
      n += 1 + (ar ? 1 : 0);
      continue;
    }
    const int f = (G.nflat_interior > 0) + (G.nflat > G.nflat_interior);
    n += f * (2 + (ax ? 1 : 0) + (ar ? 2 : 0) + (mw ? 1 : 0));
  }
  return n;
}

int qds_set_step_mode(qds_handle *h, int mode) {
  if (!h) return fail(QDS_ERR_INVALID_ARG, "NULL handle");
  if (mode < QDS_STEP_DEFAULT || mode > QDS_STEP_MARCH) return fail(QDS_ERR_INVALID_ARG, "unknown step mode");
  h->mode = mode;
  drop_graphs(h);
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
                                                   p.n_modes, p.nx, p.nr, row_ld(p), s_ax, s_ar);
  else
    import_kernel<double><<<592, kThreads, 0, st>>>((const double2 *)src, (C<double> *)b, (C<double> *)(b + half),
                                                    p.n_modes, p.nx, p.nr, row_ld(p), s_ax, s_ar);
  CU(cudaGetLastError());
  reset_kernel<<<1, 32, 0, st>>>(h->d_ctrl);
  CU(cudaGetLastError());
  h->host_step = 0;
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
                                                   (double2 *)dst, p.n_modes, p.nx, p.nr, row_ld(p), p.flags, s_ax, s_ar);
  else
    export_kernel<double><<<592, kThreads, 0, st>>>((const C<double> *)b, (const C<double> *)(b + half), h->d_ctrl,
                                                    (double2 *)dst, p.n_modes, p.nx, p.nr, row_ld(p), p.flags, s_ax,
                                                    s_ar);
  CU(cudaGetLastError());
  return QDS_OK;
}

int qds_get_state(qds_handle *h, void *dst, void *stream) { return qds_get_state_i(h, 0, dst, stream); }

int qds_set_sources_i(qds_handle *h, int i, const qds_sources *src, long long stride, void *stream) {
  if (!h || i < 0 || i >= h->n_inst) return fail(QDS_ERR_INVALID_ARG, "bad handle or instance");
  if (stride < 0) return fail(QDS_ERR_INVALID_ARG, "negative source stride");
  if (sources_equal(h, i, src, stride)) return QDS_OK;
  if (h->fp32) set_sources_i<float>(h, i, src, stride);
  else set_sources_i<double>(h, i, src, stride);
  return upload_inst(h, (cudaStream_t)stream);
}

int qds_set_inflow_i(qds_handle *h, int i, const void *tr_plus_dev, const void *tth_minus_dev, long long stride,
                     void *stream) {
  if (!h || i < 0 || i >= h->n_inst) return fail(QDS_ERR_INVALID_ARG, "bad handle or instance");
  if (stride < 0) return fail(QDS_ERR_INVALID_ARG, "negative inflow stride");
  if ((tr_plus_dev || tth_minus_dev) && (h->params[i].flags & QDS_X_PERIODIC))
    return fail(QDS_ERR_INVALID_ARG, "injection at x_min needs an open x boundary");
  if (h->fp32) set_inflow_i<float>(h, i, tr_plus_dev, tth_minus_dev, stride);
  else set_inflow_i<double>(h, i, tr_plus_dev, tth_minus_dev, stride);
  return upload_inst(h, (cudaStream_t)stream);
}

int qds_step(qds_handle *h, const qds_sources *src, int nsteps, void *stream) {
  if (!h) return fail(QDS_ERR_INVALID_ARG, "NULL handle");
  if (nsteps < 0) return fail(QDS_ERR_INVALID_ARG, "nsteps < 0");
  if (nsteps == 0) return QDS_OK;
  cudaStream_t st = (cudaStream_t)stream;
  if (src) {
    // constant sources for this call (every instance of a batch: none)
    const bool any = src->jx || src->jr || src->jth || src->s_ext;
    if (any && h->n_inst != 1)
      return fail(QDS_ERR_UNSUPPORTED, "a batch takes per-instance sources (qds_set_sources_i)");
    bool same = true;
    for (int i = 0; i < h->n_inst; i++) same = same && sources_equal(h, i, any ? src : nullptr, 0);
    if (!same) {
      for (int i = 0; i < h->n_inst; i++) {
        if (h->fp32) set_sources_i<float>(h, i, any ? src : nullptr, 0);
        else set_sources_i<double>(h, i, any ? src : nullptr, 0);
      }
      int rc = upload_inst(h, st);
      if (rc) return rc;
    }
  }
  h->host_step += (unsigned long long)nsteps;
  // per-step sources: the steps of this call count from here
  if (any_strided(h)) {
    src_base_kernel<<<1, 32, 0, st>>>(h->d_ctrl);
    CU(cudaGetLastError());
  }
  // Multi-step calls replay a captured graph of G steps.
  const int G = 16;
  if (nsteps < G) {
    cudaError_t e = launch_steps(h, nsteps, st);
    if (e != cudaSuccess) return fail(QDS_ERR_CUDA, std::string("step launch: ") + cudaGetErrorString(e));
    return QDS_OK;
  }
  auto key = std::make_tuple(G, (void *)st);
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

size_t qds_working_bytes(const qds_handle *h, int i) {
  if (!h || i < 0 || i >= h->n_inst) return 0;
  return half_bytes(h->params[i]);
}

unsigned long long qds_steps_taken(const qds_handle *h) { return h ? h->host_step : 0; }

int qds_save_working(qds_handle *h, int i, void *dst_dev, size_t bytes, void *stream) {
  if (!h || !dst_dev || i < 0 || i >= h->n_inst) return fail(QDS_ERR_INVALID_ARG, "bad handle, instance or destination");
  const size_t hb = half_bytes(h->params[i]);
  const size_t n = bytes < hb ? bytes : hb;  // a prefix (the EM planes lead) or the whole state
  const char *src = h->state + h->inst_off[i] + (h->host_step & 1ull) * hb;
  CU(cudaMemcpyAsync(dst_dev, src, n, cudaMemcpyDeviceToDevice, (cudaStream_t)stream));
  return QDS_OK;
}

int qds_restore_working(qds_handle *h, const void *src_dev, size_t bytes, unsigned long long step, void *stream) {
  if (!h || !src_dev) return fail(QDS_ERR_INVALID_ARG, "bad handle or source");
  if (h->n_inst != 1) return fail(QDS_ERR_UNSUPPORTED, "restoring a working snapshot needs a single-instance handle");
  const size_t hb = half_bytes(h->params[0]);
  if (bytes < hb) return fail(QDS_ERR_INVALID_ARG, "working snapshot buffer too small (qds_working_bytes)");
  cudaStream_t st = (cudaStream_t)stream;
  CU(cudaMemcpyAsync(h->state + h->inst_off[0] + (step & 1ull) * hb, src_dev, hb, cudaMemcpyDeviceToDevice, st));
  set_step_kernel<<<1, 32, 0, st>>>(h->d_ctrl, step);
  CU(cudaGetLastError());
  h->host_step = step;
  return QDS_OK;
}

int qds_status(qds_handle *h, void *stream) {
  if (!h) return fail(QDS_ERR_INVALID_ARG, "NULL handle");
  return read_status(h, (cudaStream_t)stream);
}

int qds_test_withhold_copy(qds_handle *h, int on, void *stream) {
  if (!h) return fail(QDS_ERR_INVALID_ARG, "NULL handle");
  set_test_kernel<<<1, 32, 0, (cudaStream_t)stream>>>(h->d_ctrl, on ? 1u : 0u);
  CU(cudaGetLastError());
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
  const int ld = row_ld(p);
  if (h->fp32)
    diag_partial_kernel<float><<<h->diag_blocks, kThreads, 0, st>>>((const C<float> *)b, (const C<float> *)(b + half),
                                                                    h->d_ctrl, p.n_modes, p.nx, p.nr, ld, p.dr,
                                                                    p.m_a * p.m_a, h->d_partial);
  else
    diag_partial_kernel<double><<<h->diag_blocks, kThreads, 0, st>>>((const C<double> *)b, (const C<double> *)(b + half),
                                                                     h->d_ctrl, p.n_modes, p.nx, p.nr, ld, p.dr,
                                                                     p.m_a * p.m_a, h->d_partial);
  CU(cudaGetLastError());
  diag_final_kernel<<<1, 32, 0, st>>>(h->d_partial, h->diag_blocks, pref, g2, g2 * g2, g2, h->d_diag, h->d_ctrl);
  CU(cudaGetLastError());
  if (profile_dev) {
    if (h->fp32)
      profile_kernel<float><<<p.nx, kThreads, 0, st>>>((const C<float> *)b, (const C<float> *)(b + half), h->d_ctrl,
                                                       p.n_modes, p.nx, p.nr, ld, p.dr, p.flags, profile_dev);
    else
      profile_kernel<double><<<p.nx, kThreads, 0, st>>>((const C<double> *)b, (const C<double> *)(b + half), h->d_ctrl,
                                                        p.n_modes, p.nx, p.nr, ld, p.dr, p.flags, profile_dev);
    CU(cudaGetLastError());
  }
  CU(cudaMemcpyAsync(out_host, h->d_diag, sizeof(double) * 4, cudaMemcpyDeviceToHost, st));
  return read_status(h, st);
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
                                                                  h->n_inst, out_dev, h->d_ctrl);
  CU(cudaGetLastError());
  return QDS_OK;
}

}  // extern "C"
