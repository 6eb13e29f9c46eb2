// qds_kernels.cuh -- CUDA kernels of the QDS library: the pass-mode stage
// kernels, the step-counter advance, state import/export and the
// diagnostics reductions.
#pragma once

#include <cuda_runtime.h>

#include "qds_stages.cuh"

namespace qds {

struct Ctrl {
  unsigned long long step;      // steps taken since the last state import
  unsigned int err;             // device-side error flags (kErr*)
  unsigned int test;            // test hook: bit 0 withholds the first bulk copy of each x-marching CTA
  unsigned long long src_base;  // step count when the current qds_step call began
};

// Sources of the current step: the descriptor's arrays advanced by the
// steps taken in this call times the per-step stride.
template <class R>
__device__ __forceinline__ const C<R> *step_src(const C<R> *a, const Inst<R> &I, const Ctrl *ctrl) {
  if (!a || I.sstride == 0) return a;
  return a + (long long)(ctrl->step - ctrl->src_base) * I.sstride;
}

// Injection arrays of the current step (null when not injecting).
template <class R>
__device__ __forceinline__ const C<R> *step_inflow(const C<R> *a, const Inst<R> &I, const Ctrl *ctrl) {
  if (!a || I.istride == 0) return a;
  return a + (long long)(ctrl->step - ctrl->src_base) * I.istride;
}

// Per-instance prefactors of the energies (diag_final_all_kernel).
struct Scal4 {
  double x, y, z, w;
};

// Device error bits in Ctrl::err
constexpr unsigned kErrTimeout = 1u;    // a bounded wait of a step kernel ran out
constexpr unsigned kErrNonfinite = 2u;  // a NaN or Inf reached the state


// Pass-mode view of the point (x0 = td.y, r0 = td.z) of instance td.x at
// step n.
template <class R, int M, bool FAST>
__device__ __forceinline__ Tile<R, M, FAST> pass_tile(const Inst<R> &I, int4 td, const Ctrl *ctrl) {
  const unsigned long long n = ctrl->step;
  Tile<R, M, FAST> t;
  t.bind(I, &I);
  t.jx = step_src(I.jx, I, ctrl);
  t.jr = step_src(I.jr, I, ctrl);
  t.jt = step_src(I.jt, I, ctrl);
  t.sext = step_src(I.sext, I, ctrl);
  t.in_rp = step_inflow(I.in_rp, I, ctrl);
  t.in_tm = step_inflow(I.in_tm, I, ctrl);
  t.nx = I.nx;
  t.nr = I.nr;
  t.ld = I.ld;
  t.J = I.nr - 1;
  t.x0 = td.y;
  t.r0 = td.z;
  t.per = (I.flags & F_X_PERIODIC) != 0;
  t.closed = (I.flags & F_R_CLOSED) != 0;
  t.mw = (I.flags & F_MOVING_WINDOW) != 0;
  t.s = t.mw ? (int)(n % (unsigned long long)I.nx) : 0;
  t.P = plane_elems(M, I.nx, I.ld);
  const int par = (int)(n & 1ull);
  t.o = I.state[par];
  t.n = I.state[par ^ 1];
  t.h = I.h;
  t.dr = I.dr;
  t.ih = I.inv_h;
  t.idr = I.inv_dr;
  t.scr = I.scratch;
  return t;
}

// Stage pass over a flat range of points: block td covers points
// td.y .. td.y + td.z - 1 of instance td.x in (x, r) order (r fastest), one
// point per thread, so no lane idles on rows beyond nr.
//
// FAST: the block list holds only blocks whose x-halo lies inside the window
// (checks skipped).  The heavy stages (axion source and current) keep more
// registers; the light ones run more CTAs per SM.
template <class R, int M, int ST, bool FAST>
__device__ __forceinline__ void flat_point(const Inst<R> *__restrict__ insts, int4 td, const Ctrl *__restrict__ ctrl) {
  if ((int)threadIdx.x >= td.z) return;
  const Inst<R> &I = insts[td.x];
  const int q = td.y + (int)threadIdx.x;
  const int w = q / I.nr, j = q - w * I.nr;
  Tile<R, M, FAST> t = pass_tile<R, M, FAST>(I, make_int4(td.x, w, j, 0), ctrl);
  run_stage<R, M, FAST>(t, ST);
}

template <int M, int ST>
constexpr int flat_ctas_per_sm() {
  return (ST == ST_SOURCE || ST == ST_CURRENT) ? (M <= 3 ? 4 : 3) : ST == ST_LEAP0 ? 5 : 6;
}

template <class R, int M, int ST, bool FAST>
__global__ void __launch_bounds__(256, flat_ctas_per_sm<M, ST>())
    flat_pass_kernel(const Inst<R> *__restrict__ insts, const int4 *__restrict__ tiles,
                     const Ctrl *__restrict__ ctrl) {
  flat_point<R, M, ST, FAST>(insts, tiles[blockIdx.x], ctrl);
}

static __global__ void advance_kernel(Ctrl *ctrl, int nsteps) {
  if (threadIdx.x == 0 && blockIdx.x == 0) ctrl->step += (unsigned long long)nsteps;
}

static __global__ void reset_kernel(Ctrl *ctrl) {
  if (threadIdx.x == 0 && blockIdx.x == 0) { ctrl->step = 0; ctrl->err = 0; }
}

// restore the step counter with a working snapshot (clears the error bits)
static __global__ void set_step_kernel(Ctrl *ctrl, unsigned long long step) {
  if (threadIdx.x == 0 && blockIdx.x == 0) { ctrl->step = step; ctrl->err = 0; }
}

static __global__ void src_base_kernel(Ctrl *ctrl) {
  if (threadIdx.x == 0 && blockIdx.x == 0) ctrl->src_base = ctrl->step;
}

static __global__ void set_test_kernel(Ctrl *ctrl, unsigned int bits) {
  if (threadIdx.x == 0 && blockIdx.x == 0) ctrl->test = bits;
}

// Canonical complex128 layout <-> working storage (precision, row stride,
// ring offset, 1/g scaling of the axion and regenerated groups).  The import
// walks the working layout so that the padding rows are written as zero.
template <class R>
__global__ void import_kernel(const double2 *__restrict__ src, C<R> *b0, C<R> *b1, int M, int nx, int nr, int ld,
                              double s_ax, double s_ar) {
  const size_t P = plane_elems(M, nx, ld), Pc = plane_elems(M, nx, nr);
  const size_t total = state_elems(M, nx, ld);
  for (size_t q = blockIdx.x * (size_t)blockDim.x + threadIdx.x; q < total; q += (size_t)gridDim.x * blockDim.x) {
    double sc = 1.0;
    C<R> z = zero<R>();
    if (q < (size_t)NFIELD * P) {
      const int f = (int)(q / P);
      if (f == PHI || f == TAP || f == TAM) sc = s_ax;
      else if (f >= TRP1) sc = s_ar;
      const size_t rem = q - (size_t)f * P;
      const int j = (int)(rem % ld);
      if (j < nr) {
        const double2 v = src[(size_t)f * Pc + (rem / ld) * nr + j];
        z = mk<R>((R)(v.x * sc), (R)(v.y * sc));
      }
    } else {
      const double2 v = src[(size_t)NFIELD * Pc + (q - (size_t)NFIELD * P)];  // phi_prev
      z = mk<R>((R)(v.x * s_ax), (R)(v.y * s_ax));
    }
    b0[q] = z;
    b1[q] = z;
  }
}

template <class R>
__global__ void export_kernel(const C<R> *__restrict__ b0, const C<R> *__restrict__ b1, const Ctrl *ctrl,
                              double2 *dst, int M, int nx, int nr, int ld, uint32_t flags, double s_ax, double s_ar) {
  const unsigned long long n = ctrl->step;
  const C<R> *b = (n & 1ull) ? b1 : b0;
  const int s = (flags & F_MOVING_WINDOW) ? (int)(n % (unsigned long long)nx) : 0;
  const size_t P = plane_elems(M, nx, ld), Pc = plane_elems(M, nx, nr);
  const size_t total = state_elems(M, nx, nr);
  for (size_t q = blockIdx.x * (size_t)blockDim.x + threadIdx.x; q < total; q += (size_t)gridDim.x * blockDim.x) {
    double sc = 1.0;
    size_t from;
    if (q < (size_t)NFIELD * Pc) {
      int f = (int)(q / Pc);
      if (f == PHI || f == TAP || f == TAM) sc = s_ax;
      else if (f >= TRP1) sc = s_ar;
      size_t rem = q % Pc;
      int j = (int)(rem % nr);
      size_t kw = rem / nr;
      int w = (int)(kw % nx), k = (int)(kw / nx);
      int sl = w + s; if (sl >= nx) sl -= nx;
      from = (size_t)f * P + ((size_t)k * nx + sl) * ld + j;
    } else {
      sc = s_ax;
      size_t rem = q - (size_t)NFIELD * Pc;
      int w = (int)(rem % nx), k = (int)(rem / nx);
      int sl = w + s; if (sl >= nx) sl -= nx;
      from = (size_t)NFIELD * P + (size_t)k * nx + sl;
    }
    C<R> z = b[from];
    dst[q] = make_double2((double)z.re * sc, (double)z.im * sc);
  }
}

// ---------------------------------------------------------------------------
// Diagnostics: energies with the azimuthal weights of Eq. fourier_decomp
// (w_0 = 1, w_m = 1/2) and the cell volume 2 pi r dr h (r_0 -> dr/8 on the
// axis row), accumulated in FP64 with Neumaier compensation.
// ---------------------------------------------------------------------------
struct Neu {
  double s = 0.0, c = 0.0;
  __device__ void add(double x) {
    double t = s + x;
    if (fabs(s) >= fabs(x)) c += (s - t) + x;
    else c += (x - t) + s;
    s = t;
  }
  __device__ double val() const { return s + c; }
};

// Compensated (Neumaier) running sum in the working precision R; the
// per-thread sums are then combined in FP64.
template <class R>
struct NeuR {
  R s = R(0), c = R(0);
  __device__ void add(R x) {
    R t = s + x;
    if (fabs(s) >= fabs(x)) c += (s - t) + x;
    else c += (x - t) + s;
    s = t;
  }
  __device__ double val() const { return (double)s + (double)c; }
};

template <class R>
__device__ __forceinline__ R nrmR(C<R> a) { return a.re * a.re + a.im * a.im; }
template <class R>
__device__ __forceinline__ R dotR(C<R> a, C<R> b) { return a.re * b.re + a.im * b.im; }

// Energy densities of one (mode, x, r) element of one instance, added to the
// four accumulators em0, axion, em1, cross (without the common prefactor).
template <class R>
__device__ __forceinline__ void diag_element(const C<R> *S, size_t P, size_t q, int nx, int nr, int ld, R dr,
                                             R ma2, NeuR<R> &a0, NeuR<R> &a1, NeuR<R> &a2, NeuR<R> &a3) {
  const int j = (int)(q % ld);
  if (j >= nr) return;  // padding row
  const int k = (int)(q / ((size_t)nx * ld));
  const R wm = k == 0 ? R(1) : R(0.5);
  const R rh = (R(j) + R(0.5)) * dr, rs = j == 0 ? dr / R(8) : R(j) * dr;
  R e[2];
  C<R> er[2], bt[2], et[2], br[2], ex[2], bx[2];
  for (int gi = 0; gi < 2; gi++) {
    const int o = gi ? TRP1 : TRP;
    C<R> tp = S[(size_t)(o + 0) * P + q], tm = S[(size_t)(o + 1) * P + q];
    C<R> up = S[(size_t)(o + 2) * P + q], um = S[(size_t)(o + 3) * P + q];
    er[gi] = R(0.5) * (tp + tm); bt[gi] = R(0.5) * (tp - tm);
    et[gi] = R(0.5) * (up + um); br[gi] = R(0.5) * (up - um);
    ex[gi] = S[(size_t)(o + 4) * P + q]; bx[gi] = S[(size_t)(o + 5) * P + q];
    e[gi] = rh * (nrmR(er[gi]) + nrmR(bt[gi])) + rs * (nrmR(et[gi]) + nrmR(br[gi])) + rs * nrmR(ex[gi]) + rh * nrmR(bx[gi]);
  }
  a0.add(wm * e[0]);
  a2.add(wm * e[1]);
  C<R> ph = S[(size_t)PHI * P + q], ap = S[(size_t)TAP * P + q], am = S[(size_t)TAM * P + q];
  R ua = rh * R(0.5) * (nrmR(ap) + nrmR(am)) + rh * (R(k * k) / (rh * rh) + ma2) * nrmR(ph);
  if (j > 0) {
    C<R> d = S[(size_t)PHI * P + q] - S[(size_t)PHI * P + q - 1];
    ua += (R(j) * dr) * nrmR(d) / (dr * dr);
  }
  a1.add(wm * ua);
  R cr = rh * (dotR(er[0], er[1]) + dotR(bt[0], bt[1])) + rs * (dotR(et[0], et[1]) + dotR(br[0], br[1])) +
         rs * dotR(ex[0], ex[1]) + rh * dotR(bx[0], bx[1]);
  a3.add(wm * cr);
}

template <class A>
__device__ __forceinline__ void block_reduce4(A &a0, A &a1, A &a2, A &a3, double *dst) {
  __shared__ double red[4][256];
  red[0][threadIdx.x] = a0.val();
  red[1][threadIdx.x] = a1.val();
  red[2][threadIdx.x] = a2.val();
  red[3][threadIdx.x] = a3.val();
  __syncthreads();
  for (int w = blockDim.x / 2; w > 0; w >>= 1) {
    if (threadIdx.x < w)
      for (int c = 0; c < 4; c++) red[c][threadIdx.x] += red[c][threadIdx.x + w];
    __syncthreads();
  }
  if (threadIdx.x == 0)
    for (int c = 0; c < 4; c++) dst[c] = red[c][0];
}

// partial[b*4 + 0..3]: em0, axion, em1, cross of one instance
template <class R>
__global__ void diag_partial_kernel(const C<R> *__restrict__ b0, const C<R> *__restrict__ b1, const Ctrl *ctrl,
                                    int M, int nx, int nr, int ld, double dr, double ma2, double *partial) {
  const C<R> *S = (ctrl->step & 1ull) ? b1 : b0;
  const size_t P = plane_elems(M, nx, ld);
  NeuR<R> a0, a1, a2, a3;
  for (size_t q = blockIdx.x * (size_t)blockDim.x + threadIdx.x; q < P; q += (size_t)gridDim.x * blockDim.x)
    diag_element<R>(S, P, q, nx, nr, ld, (R)dr, (R)ma2, a0, a1, a2, a3);
  block_reduce4(a0, a1, a2, a3, partial + blockIdx.x * 4);
}

// All instances of a batch in one launch: grid (blocks, instances).
template <class R>
__global__ void diag_partial_all_kernel(const Inst<R> *__restrict__ insts, const Ctrl *ctrl, double *partial) {
  const Inst<R> &I = insts[blockIdx.y];
  const C<R> *S = I.state[ctrl->step & 1ull];
  const size_t P = plane_elems(I.M, I.nx, I.ld);
  NeuR<R> a0, a1, a2, a3;
  for (size_t q = blockIdx.x * (size_t)blockDim.x + threadIdx.x; q < P; q += (size_t)gridDim.x * blockDim.x)
    diag_element<R>(S, P, q, I.nx, I.nr, I.ld, I.dr, I.ma2, a0, a1, a2, a3);
  block_reduce4(a0, a1, a2, a3, partial + ((size_t)blockIdx.y * gridDim.x + blockIdx.x) * 4);
}

// scal[i] = {pi dr dx, g^2 or 1, g^4 or 1, g^2 or 1} per instance; a
// non-finite energy sets kErrNonfinite
static __global__ void diag_final_all_kernel(const double *partial, int nblk, const Scal4 *scal, int n, double *out,
                                             Ctrl *ctrl) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  Neu s[4];
  for (int b = 0; b < nblk; b++)
    for (int c = 0; c < 4; c++) s[c].add(partial[((size_t)i * nblk + b) * 4 + c]);
  const Scal4 f = scal[i];
  out[4 * i + 0] = f.x * s[0].val();
  out[4 * i + 1] = f.x * s[1].val() * f.y;
  out[4 * i + 2] = f.x * s[2].val() * f.z;
  out[4 * i + 3] = 2.0 * f.x * s[3].val() * f.w;
  bool ok = true;
  for (int c = 0; c < 4; c++) ok = ok && isfinite(out[4 * i + c]);
  if (!ok) atomicOr(&ctrl->err, kErrNonfinite);
}

static __global__ void diag_final_kernel(const double *partial, int nblk, double pref, double s_ax2, double s_ar2,
                                         double s_cross, double *out, Ctrl *ctrl) {
  if (threadIdx.x != 0 || blockIdx.x != 0) return;
  Neu s[4];
  for (int b = 0; b < nblk; b++)
    for (int c = 0; c < 4; c++) s[c].add(partial[b * 4 + c]);
  out[0] = pref * s[0].val();
  out[1] = pref * s[1].val() * s_ax2;
  out[2] = pref * s[2].val() * s_ar2;
  out[3] = 2.0 * pref * s[3].val() * s_cross;
  if (!(isfinite(out[0]) && isfinite(out[1]) && isfinite(out[2]) && isfinite(out[3]))) atomicOr(&ctrl->err, kErrNonfinite);
}

// U(x_w) = int (1/2)(|E_perp|^2 + |B_perp|^2) dA of group 0 (Sec. 4.1), one
// block per window column.
template <class R>
__global__ void profile_kernel(const C<R> *__restrict__ b0, const C<R> *__restrict__ b1, const Ctrl *ctrl,
                               int M, int nx, int nr, int ld, double dr, uint32_t flags, double *prof) {
  const unsigned long long n = ctrl->step;
  const C<R> *S = (n & 1ull) ? b1 : b0;
  const int s = (flags & F_MOVING_WINDOW) ? (int)(n % (unsigned long long)nx) : 0;
  const int w = blockIdx.x;
  int sl = w + s; if (sl >= nx) sl -= nx;
  const size_t P = plane_elems(M, nx, ld);
  Neu acc;
  for (int q = threadIdx.x; q < M * nr; q += blockDim.x) {
    const int k = q / nr, j = q % nr;
    const size_t e = ((size_t)k * nx + sl) * ld + j;
    C<R> tp = S[(size_t)TRP * P + e], tm = S[(size_t)TRM * P + e];
    C<R> up = S[(size_t)TTP * P + e], um = S[(size_t)TTM * P + e];
    const double wm = k == 0 ? 1.0 : 0.5;
    const double rh = (j + 0.5) * dr, rs = j == 0 ? dr / 8.0 : j * dr;
    acc.add(wm * (rh * ((double)nrmR(R(0.5) * (tp + tm)) + (double)nrmR(R(0.5) * (tp - tm))) +
                  rs * ((double)nrmR(R(0.5) * (up + um)) + (double)nrmR(R(0.5) * (up - um)))));
  }
  __shared__ double red[256];
  red[threadIdx.x] = acc.val();
  __syncthreads();
  for (int k = blockDim.x / 2; k > 0; k >>= 1) {
    if (threadIdx.x < k) red[threadIdx.x] += red[threadIdx.x + k];
    __syncthreads();
  }
  if (threadIdx.x == 0) prof[w] = 3.14159265358979323846 * dr * red[0];
}

}  // namespace qds
