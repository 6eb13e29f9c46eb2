// qds_adjoint.cu -- qds_adjoint_step(): one transposed step of the EM group
// and the axion on the GPU (the transpose in qds_adjoint.cuh, one kernel per
// transposed pass, one thread per (x, r) point of the window).
//
// The caller passes the forward state at the start of the step and the
// adjoint of the state after it, both in the canonical complex128 layout in
// physical variables (what qds_get_state returns), and gets the adjoint of
// the state before the step in place.  The transpose runs in the handle's
// working precision; with QDS_FP32 the state and adjoint are converted to
// complex64 (no 1/g scaling: the adjoint has no weak-coupling cancellation).
#include <cuda_runtime.h>

#include <cstring>
#include <string>

#include "../../include/qds.h"
#include "qds_adjoint.cuh"

using namespace qds;

// defined in qds_api.cu
void qds_internal_set_error(const std::string &m);
int qds_internal_params(const qds_handle *h, int i, qds_params *out);
int qds_internal_layout(const qds_handle *h, int i, int *ld);

namespace {

int fail_ad(int code, const std::string &m) {
  qds_internal_set_error(m);
  return code;
}

constexpr int kThr = 256;
size_t up256(size_t x) { return (x + 255) / 256 * 256; }

// work layout: [a descriptor-sized slot, unused] [N_SB scratch planes] [lambda^(n+1) copy]
//              FP32 only: [forward state] [lambda^n]
template <class R>
struct AdjLayout {
  size_t off_scr, off_ln, off_f, off_lo, total;
  AdjLayout(const qds_params &p) {
    const size_t P = plane_elems(p.n_modes, p.nx, p.nr), E = state_elems(p.n_modes, p.nx, p.nr);
    const size_t eb = sizeof(C<R>);
    off_scr = up256(sizeof(Inst<R>));
    off_ln = off_scr + up256((size_t)N_SB * P * eb);
    off_f = off_ln + up256(E * eb);
    if (sizeof(R) == 4) {
      off_lo = off_f + up256(E * eb);
      total = off_lo + up256(E * eb);
    } else {
      off_lo = off_f;
      total = off_f;
    }
  }
};

// AD_SRC: one thread per (x, r) point with all modes; AD_LEAP, AD_CELL: one
// thread per (mode, x, r), r fastest.
template <class R, int M, int ST>
__global__ void __launch_bounds__(kThr, sizeof(R) == 8 ? 1 : (ST == AD_SRC ? (M <= 3 ? 3 : 2) : 6)) adjoint_kernel(Adj<R, M> a) {
  const int n = a.nx * a.nr;
  const int total = ST == AD_SRC ? n : M * n;
  double acc = 0;
  for (int q = blockIdx.x * blockDim.x + threadIdx.x; q < total; q += gridDim.x * blockDim.x) {
    const int k = ST == AD_SRC ? 0 : q / n, p = q - k * n;
    const int w = p / a.nr, j = p - w * a.nr;
    adj_point<R, M>(a, ST, k, w, j, acc);
  }
  if (ST == AD_SRC && a.dg) {
    for (int o = 16; o > 0; o >>= 1) acc += __shfl_down_sync(0xffffffffu, acc, o);
    if ((threadIdx.x & 31) == 0 && acc != 0.0) atomicAdd(a.dg, acc);
  }
}

// Conversions between complex128 and the working precision over the part of
// a state that the transpose uses: the EM and axion fields (the first
// n_lo elements) and phi_prev (after the regenerated fields, skip elements
// further on); n counts the elements converted.
__device__ __forceinline__ size_t used_index(size_t q, size_t n_lo, size_t skip) { return q < n_lo ? q : q + skip; }

template <class R>
__global__ void to_work_kernel(const double2 *__restrict__ src, C<R> *dst, size_t n, size_t n_lo, size_t skip) {
  for (size_t q = blockIdx.x * (size_t)blockDim.x + threadIdx.x; q < n; q += (size_t)gridDim.x * blockDim.x) {
    const size_t i = used_index(q, n_lo, skip);
    double2 v = src[i];
    dst[i] = mk<R>((R)v.x, (R)v.y);
  }
}

template <class R>
__global__ void from_work_kernel(const C<R> *__restrict__ src, double2 *dst, size_t n, size_t n_lo, size_t skip) {
  for (size_t q = blockIdx.x * (size_t)blockDim.x + threadIdx.x; q < n; q += (size_t)gridDim.x * blockDim.x) {
    const size_t i = used_index(q, n_lo, skip);
    C<R> v = src[i];
    dst[i] = make_double2((double)v.re, (double)v.im);
  }
}

template <class R, int M>
cudaError_t launch_all(Adj<R, M> a, int blocks, cudaStream_t st) {
  adjoint_kernel<R, M, AD_SRC><<<blocks, kThr, 0, st>>>(a);
  adjoint_kernel<R, M, AD_LEAP><<<M * blocks, kThr, 0, st>>>(a);
  adjoint_kernel<R, M, AD_CELL><<<M * blocks, kThr, 0, st>>>(a);
  return cudaGetLastError();
}

// F: the forward state at the start of the step, with row stride ld and
// ring offset s (the canonical layout: ld = nr, s = 0; a working snapshot:
// the handle's row stride and the window's offset at that step).
template <class R, int M>
Adj<R, M> make_adj(const qds_params &p, const Inst<R> &h_inst, const Inst<R> *d_inst, const C<R> *F,
                   const C<R> *LN, C<R> *LO, C<R> *SB, double *dg, bool zero_regen, int ld = 0, int s = 0,
                   const C<R> *Fnext = nullptr) {
  Adj<R, M> a;
  std::memset(&a, 0, sizeof a);
  const int nx = p.nx, nr = p.nr;
  const size_t P = plane_elems(M, nx, nr);
  if (ld == 0) ld = nr;
  Tile<R, M, false> &t = a.f;
  t.bind(h_inst, d_inst);
  t.nx = nx; t.nr = nr; t.ld = ld; t.J = nr - 1; t.x0 = 0; t.r0 = 0; t.s = s;
  t.per = false; t.closed = false; t.mw = false;
  t.P = plane_elems(M, nx, ld); t.o = F; t.n = nullptr;
  t.h = (R)p.dx; t.dr = (R)p.dr; t.ih = (R)(1.0 / p.dx); t.idr = (R)(1.0 / p.dr);
  t.scr = nullptr;
  t.cw = -(1 << 28);  // each point sets the column cache (adjoint_kernel)
  a.fnext = Fnext;
  a.ln = LN; a.lo = LO; a.sb = SB; a.dg = dg;
  a.nx = nx; a.nr = nr; a.J = nr - 1; a.P = (unsigned)P;
  a.mw = (p.flags & QDS_MOVING_WINDOW) != 0;
  a.zero_regen = zero_regen;
  a.h = t.h; a.dr = t.dr; a.ih = t.ih; a.idr = t.idr;
  a.gs = (R)p.g; a.ma2 = (R)(p.m_a * p.m_a);
  a.set_consts();
  return a;
}

template <class R>
int adjoint(const qds_params &p, const qds_sources *src, const void *fwd, void *adj, void *work, size_t work_bytes,
            double *dg, cudaStream_t st) {
  AdjLayout<R> L(p);
  if (work_bytes < L.total) return fail_ad(QDS_ERR_INVALID_ARG, "adjoint work buffer too small");
  if (reinterpret_cast<uintptr_t>(work) % 256) return fail_ad(QDS_ERR_INVALID_ARG, "adjoint work buffer must be 256-byte aligned");
  const int M = p.n_modes, nx = p.nx, nr = p.nr;
  const size_t E = state_elems(M, nx, nr);
  char *b = static_cast<char *>(work);
  Inst<R> I;
  std::memset(&I, 0, sizeof I);
  I.nx = nx; I.nr = nr; I.ld = nr; I.M = M; I.flags = p.flags;
  I.h = (R)p.dx; I.dr = (R)p.dr; I.inv_h = (R)(1.0 / p.dx); I.inv_dr = (R)(1.0 / p.dr);
  I.ma2 = (R)(p.m_a * p.m_a);
  I.gs = (R)p.g; I.gj = (R)p.g;
  if (src) {
    I.jx = (const C<R> *)src->jx;
    I.jt = (const C<R> *)src->jth;
    I.sext = (const C<R> *)src->s_ext;
  }
  // the passes take the descriptor's values by argument: no device copy
  cudaError_t e = cudaSuccess;
  C<R> *SB = reinterpret_cast<C<R> *>(b + L.off_scr);
  C<R> *LN = reinterpret_cast<C<R> *>(b + L.off_ln);
  const C<R> *F;
  C<R> *LO;
  const int cblocks = 1184;
  // the regenerated fields (TRP1 .. BX1) are neither read nor needed
  const size_t P = plane_elems(M, nx, nr), n_lo = (size_t)TRP1 * P, skip = (size_t)(NFIELD - TRP1) * P;
  const size_t n_used = E - skip;
  if (sizeof(R) == 4) {
    C<R> *Fw = reinterpret_cast<C<R> *>(b + L.off_f);
    to_work_kernel<R><<<cblocks, kThr, 0, st>>>((const double2 *)fwd, Fw, n_used, n_lo, skip);
    to_work_kernel<R><<<cblocks, kThr, 0, st>>>((const double2 *)adj, LN, n_used, n_lo, skip);
    F = Fw;
    LO = reinterpret_cast<C<R> *>(b + L.off_lo);
  } else {
    if ((e = cudaMemcpyAsync(LN, adj, n_lo * sizeof(C<R>), cudaMemcpyDeviceToDevice, st)) != cudaSuccess ||
        (e = cudaMemcpyAsync(LN + n_lo + skip, static_cast<const C<R> *>(adj) + n_lo + skip,
                             (E - n_lo - skip) * sizeof(C<R>), cudaMemcpyDeviceToDevice, st)) != cudaSuccess)
      return fail_ad(QDS_ERR_CUDA, std::string("adjoint copy: ") + cudaGetErrorString(e));
    F = static_cast<const C<R> *>(fwd);
    LO = static_cast<C<R> *>(adj);
  }
  const Inst<R> *d_inst = reinterpret_cast<const Inst<R> *>(b);
  const int blocks = (int)((size_t(nx) * nr + kThr - 1) / kThr);
  switch (M) {
    case 1: e = launch_all<R, 1>(make_adj<R, 1>(p, I, d_inst, F, LN, LO, SB, dg, sizeof(R) == 8), blocks, st); break;
    case 2: e = launch_all<R, 2>(make_adj<R, 2>(p, I, d_inst, F, LN, LO, SB, dg, sizeof(R) == 8), blocks, st); break;
    case 3: e = launch_all<R, 3>(make_adj<R, 3>(p, I, d_inst, F, LN, LO, SB, dg, sizeof(R) == 8), blocks, st); break;
    case 4: e = launch_all<R, 4>(make_adj<R, 4>(p, I, d_inst, F, LN, LO, SB, dg, sizeof(R) == 8), blocks, st); break;
    default: e = cudaErrorInvalidValue;
  }
  if (e != cudaSuccess) return fail_ad(QDS_ERR_CUDA, std::string("adjoint launch: ") + cudaGetErrorString(e));
  if (sizeof(R) == 4) {
    from_work_kernel<R><<<cblocks, kThr, 0, st>>>(LO, (double2 *)adj, n_used, n_lo, skip);
    if ((e = cudaGetLastError()) != cudaSuccess ||
        (e = cudaMemsetAsync(static_cast<double2 *>(adj) + n_lo, 0, skip * sizeof(double2), st)) != cudaSuccess)
      return fail_ad(QDS_ERR_CUDA, std::string("adjoint export: ") + cudaGetErrorString(e));
  }
  return QDS_OK;
}

// The transposed step in the working precision without conversions: the
// forward state is a working snapshot (qds_save_working) taken `step` steps
// after the state import, lam_in / lam_out canonical arrays of the working
// precision (distinct buffers).  Work: the descriptor and the scratch planes.
size_t work_w_bytes(const qds_params &p, size_t elem) {
  return up256(sizeof(Inst<double>)) + up256((size_t)N_SB * plane_elems(p.n_modes, p.nx, p.nr) * elem);
}

template <class R>
int adjoint_w(const qds_params &p, int ld, const qds_sources *src, const void *fwd, const void *fwd_next,
              unsigned long long step, const void *lam_in, void *lam_out, void *work, size_t work_bytes, double *dg,
              cudaStream_t st) {
  if (work_bytes < work_w_bytes(p, sizeof(C<R>))) return fail_ad(QDS_ERR_INVALID_ARG, "adjoint work buffer too small");
  if (reinterpret_cast<uintptr_t>(work) % 256) return fail_ad(QDS_ERR_INVALID_ARG, "adjoint work buffer must be 256-byte aligned");
  if (lam_in == lam_out) return fail_ad(QDS_ERR_INVALID_ARG, "lam_in and lam_out must be distinct buffers");
  const int M = p.n_modes, nx = p.nx, nr = p.nr;
  char *b = static_cast<char *>(work);
  Inst<R> I;
  std::memset(&I, 0, sizeof I);
  I.nx = nx; I.nr = nr; I.ld = ld; I.M = M; I.flags = p.flags;
  I.h = (R)p.dx; I.dr = (R)p.dr; I.inv_h = (R)(1.0 / p.dx); I.inv_dr = (R)(1.0 / p.dr);
  I.ma2 = (R)(p.m_a * p.m_a);
  I.gs = (R)p.g; I.gj = (R)p.g;
  if (src) {
    I.jx = (const C<R> *)src->jx;
    I.jt = (const C<R> *)src->jth;
    I.sext = (const C<R> *)src->s_ext;
  }
  // the passes take the descriptor's values by argument: no device copy
  cudaError_t e = cudaSuccess;
  C<R> *SB = reinterpret_cast<C<R> *>(b + up256(sizeof(Inst<double>)));
  const Inst<R> *d_inst = reinterpret_cast<const Inst<R> *>(b);
  const C<R> *F = static_cast<const C<R> *>(fwd);
  const C<R> *FN = static_cast<const C<R> *>(fwd_next);
  const C<R> *LN = static_cast<const C<R> *>(lam_in);
  C<R> *LO = static_cast<C<R> *>(lam_out);
  const int s = (p.flags & QDS_MOVING_WINDOW) ? (int)(step % (unsigned long long)nx) : 0;
  const int blocks = (int)((size_t(nx) * nr + kThr - 1) / kThr);
  switch (M) {
    case 1: e = launch_all<R, 1>(make_adj<R, 1>(p, I, d_inst, F, LN, LO, SB, dg, false, ld, s, FN), blocks, st); break;
    case 2: e = launch_all<R, 2>(make_adj<R, 2>(p, I, d_inst, F, LN, LO, SB, dg, false, ld, s, FN), blocks, st); break;
    case 3: e = launch_all<R, 3>(make_adj<R, 3>(p, I, d_inst, F, LN, LO, SB, dg, false, ld, s, FN), blocks, st); break;
    case 4: e = launch_all<R, 4>(make_adj<R, 4>(p, I, d_inst, F, LN, LO, SB, dg, false, ld, s, FN), blocks, st); break;
    default: e = cudaErrorInvalidValue;
  }
  if (e != cudaSuccess) return fail_ad(QDS_ERR_CUDA, std::string("adjoint launch: ") + cudaGetErrorString(e));
  return QDS_OK;
}

}  // namespace

extern "C" size_t qds_adjoint_work_bytes_w(const qds_handle *h, int i) {
  qds_params p;
  if (qds_internal_params(h, i, &p)) return 0;
  return work_w_bytes(p, (p.flags & QDS_FP32) ? sizeof(C<float>) : sizeof(C<double>));
}

extern "C" int qds_adjoint_step_w(qds_handle *h, int i, const qds_sources *src, const void *fwd_working_dev,
                                  const void *fwd_next_dev, unsigned long long fwd_step, const void *lam_in_dev,
                                  void *lam_out_dev, void *work_dev, size_t work_bytes, double *dLdg_dev,
                                  void *stream) {
  qds_params p;
  int rc = qds_internal_params(h, i, &p);
  if (rc) return rc;
  int ld = 0;
  if ((rc = qds_internal_layout(h, i, &ld))) return rc;
  if (!fwd_working_dev || !lam_in_dev || !lam_out_dev || !work_dev)
    return fail_ad(QDS_ERR_INVALID_ARG, "NULL state, adjoint or work pointer");
  if (p.flags & (QDS_X_PERIODIC | QDS_R_CLOSED))
    return fail_ad(QDS_ERR_UNSUPPORTED, "the adjoint covers open boundaries only");
  if (!(p.flags & QDS_AXION)) return fail_ad(QDS_ERR_UNSUPPORTED, "the adjoint step needs QDS_AXION");
  cudaStream_t st = (cudaStream_t)stream;
  if (p.flags & QDS_FP32)
    return adjoint_w<float>(p, ld, src, fwd_working_dev, fwd_next_dev, fwd_step, lam_in_dev, lam_out_dev, work_dev,
                            work_bytes, dLdg_dev, st);
  return adjoint_w<double>(p, ld, src, fwd_working_dev, fwd_next_dev, fwd_step, lam_in_dev, lam_out_dev, work_dev,
                           work_bytes, dLdg_dev, st);
}

extern "C" size_t qds_adjoint_work_bytes(const qds_handle *h, int i) {
  qds_params p;
  if (qds_internal_params(h, i, &p)) return 0;
  return (p.flags & QDS_FP32) ? AdjLayout<float>(p).total : AdjLayout<double>(p).total;
}

extern "C" int qds_adjoint_step(qds_handle *h, int i, const qds_sources *src, const void *fwd_state_dev,
                                void *adj_state_dev, void *work_dev, size_t work_bytes, double *dLdg_dev,
                                void *stream) {
  qds_params p;
  int rc = qds_internal_params(h, i, &p);
  if (rc) return rc;
  if (!fwd_state_dev || !adj_state_dev || !work_dev) return fail_ad(QDS_ERR_INVALID_ARG, "NULL state, adjoint or work pointer");
  if (p.flags & (QDS_X_PERIODIC | QDS_R_CLOSED))
    return fail_ad(QDS_ERR_UNSUPPORTED, "the adjoint covers open boundaries only");
  if (!(p.flags & QDS_AXION)) return fail_ad(QDS_ERR_UNSUPPORTED, "the adjoint step needs QDS_AXION");
  cudaStream_t st = (cudaStream_t)stream;
  if (p.flags & QDS_FP32) return adjoint<float>(p, src, fwd_state_dev, adj_state_dev, work_dev, work_bytes, dLdg_dev, st);
  return adjoint<double>(p, src, fwd_state_dev, adj_state_dev, work_dev, work_bytes, dLdg_dev, st);
}
