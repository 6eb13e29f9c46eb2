// qds_stages.cuh -- the point formulas of one QDS + axion + AREM step and
// the pass-mode accessor over the whole grid.  The formulas are written
// against an accessor type TT (the pass-mode Tile below, or the x-marching
// kernels' shared-memory view in qds_march.cuh) that supplies the old state,
// the intermediate planes of the step and the sources.
//
// Window coordinates: cell w sits at x_w, face w at x_{w+1/2}; the storage
// slot of window position w is (w + s) mod nx, where s advances by one per
// step when the window moves (the x-shift of the whole box is an index
// offset, not a copy).  Outside the box (non-periodic) every field reads as
// zero, which is the open x boundary of Eq. em_x_open / axion_x_open.
#pragma once

#include "qds_common.cuh"

#if defined(QDS_EMU)
#include <cstdio>
#include <cstdlib>
#define QDS_CHECK(cond, what)                                              \
  do {                                                                     \
    if (!(cond)) {                                                         \
      std::fprintf(stderr, "qds emu bounds: %s (%s:%d)\n", what, __FILE__, \
                   __LINE__);                                              \
      std::abort();                                                        \
    }                                                                      \
  } while (0)
#else
#define QDS_CHECK(cond, what) ((void)0)
#endif

#if defined(__CUDACC__)
#define QDS_NOINL __host__ __device__ __forceinline__
#else
#define QDS_NOINL inline
#endif

namespace qds {

template <class R>
QDS_HD C<R> ldg(const C<R> *p) {
#if defined(__CUDA_ARCH__)
  if (sizeof(R) == 4) {
    float2 v = __ldg(reinterpret_cast<const float2 *>(p));
    return mk<R>((R)v.x, (R)v.y);
  } else {
    double2 v = __ldg(reinterpret_cast<const double2 *>(p));
    return mk<R>((R)v.x, (R)v.y);
  }
#else
  return *p;
#endif
}

// Pass-mode accessor: one pass per stage over the whole grid, intermediates
// in the new state buffer and the scratch planes.  FAST = true: every access
// of the point (its x-halo included) lies inside the window, so the accessors
// skip their checks (the formulas themselves only touch rows 0..nr-1).
template <class R, int M, bool FAST = false>
struct Tile {
  using Real = R;
  static constexpr int kM = M;
  static constexpr bool kSM = false;  // intermediates are global planes
  const Inst<R> *I;
  // values of the descriptor used per point, held in registers (loads
  // through I could not be hoisted past the stores of a pass)
  const C<R> *jx, *jr, *jt, *sext;
  const C<R> *in_rp, *in_tm;  // injection at x_min (may be null)
  R gs, gj, ma2;
  uint32_t flags;
  QDS_HD void bind(const Inst<R> &d, const Inst<R> *dev) {
    I = dev;
    jx = d.jx; jr = d.jr; jt = d.jt; sext = d.sext;
    in_rp = d.in_rp; in_tm = d.in_tm;
    gs = d.gs; gj = d.gj; ma2 = d.ma2;
    flags = d.flags;
  }
  int nx, nr, J;       // J = nr - 1: last integer row / last half row
  int ld;              // row stride of the working planes
  int x0, r0;          // point origin in window coordinates
  int s;               // ring offset of the window
  bool per, closed, mw;
  size_t P;            // elements per field (M planes)
  const C<R> *o;       // old state
  C<R> *n;             // new state
  R h, dr, ih, idr;
  C<R> *scr;              // scratch planes Gamma_a, j_a,x, j_a,r, j_a,th
  mutable C<R> dummy;     // target of out-of-domain accesses
#if defined(QDS_EMU)
  size_t state_len;    // bounds for the emulator
#endif

  // ---------------- index helpers ----------------
  // Element offsets within one instance fit in 32 bits (checked at create).
  // The ring slots of the columns cw-1 .. cw+2 around the point being
  // computed are cached (set_point); other columns take the general path.
  int cw;              // window position the cache refers to
  int cs0, cs1, cs2, cs3;  // slot(cw-1) .. slot(cw+2), -1 outside the window
  QDS_HD bool cell_ok(int w) const { return per || (w >= 0 && w < nx); }
  QDS_HD bool face_ok(int w) const { return per || (w >= 0 && w <= nx - 2); }
  // slot of window position w, or -1 outside the window (non-periodic)
  QDS_HD int slot_slow(int w) const {
    if (per) { w %= nx; if (w < 0) w += nx; return w; }
    if (w < 0 || w >= nx) return -1;
    int q = w + s;
    return q >= nx ? q - nx : q;
  }
  QDS_HD void set_point(int w) {
    cw = w;
    cs0 = slot_slow(w - 1);
    cs1 = slot_slow(w);
    cs2 = slot_slow(w + 1);
    cs3 = slot_slow(w + 2);
  }
  QDS_HD int slot(int w) const {
    const int d = w - cw;
    if (d == -1) return cs0;
    if (d == 0) return cs1;
    if (d == 1) return cs2;
    if (d == 2) return cs3;
    return slot_slow(w);
  }
  QDS_HD unsigned eidx(int field, int k, int sl, int j) const {
    return (unsigned)field * (unsigned)P + ((unsigned)k * (unsigned)nx + (unsigned)sl) * (unsigned)ld + (unsigned)j;
  }
  QDS_HD size_t gidx(int field, int k, int w, int j) const { return eidx(field, k, slot(w), j); }
  QDS_HD C<R> cell(int field, int k, int w, int j) const {
    const int sl = slot(w);
    if (FAST) {  // the point and its halo lie inside the window
#if defined(QDS_EMU)
      QDS_CHECK(j >= 0 && j < nr && sl >= 0, "unchecked cell access");
#endif
      return ldg(o + eidx(field, k, sl, j));
    }
    if ((unsigned)j >= (unsigned)nr) return zero<R>();
    if (sl < 0) {
      // the exterior cell behind x_min: zero (open boundary, Eq. em_x_open),
      // or the injected inflow T_r^+ / T_th^- of the EM field
      if (w == -1 && !per) {
        if (field == TRP && in_rp) return ldg(in_rp + (size_t)k * nr + j);
        if (field == TTM && in_tm) return ldg(in_tm + (size_t)k * nr + j);
      }
      return zero<R>();
    }
#if defined(QDS_EMU)
    QDS_CHECK(eidx(field, k, sl, j) < state_len, "cell read");
#endif
    return ldg(o + eidx(field, k, sl, j));
  }
  QDS_HD C<R> face(int field, int k, int w, int j) const {
    const int sl = slot(w);
    if (FAST) {
#if defined(QDS_EMU)
      QDS_CHECK(j >= 0 && j < nr && sl >= 0 && (per || w <= nx - 2), "unchecked face access");
#endif
      return ldg(o + eidx(field, k, sl, j));
    }
    if (sl < 0 || (!per && w == nx - 1) || (unsigned)j >= (unsigned)nr) return zero<R>();
#if defined(QDS_EMU)
    QDS_CHECK(eidx(field, k, sl, j) < state_len, "face read");
#endif
    return ldg(o + eidx(field, k, sl, j));
  }
  QDS_HD C<R> prev(int k, int w) const {
    if (!face_ok(w)) return zero<R>();
    return ldg(o + (size_t)NFIELD * P + (size_t)k * nx + slot(w));
  }
  // caller-owned source arrays [M][nx][nr] (native staggered positions),
  // indexed in window order (not by ring slot)
  QDS_HD C<R> srcv(const C<R> *a, int k, int w, int j) const {
    if (!a || !cell_ok(w) || j < 0 || j >= nr) return zero<R>();
    if (per) { w %= nx; if (w < 0) w += nx; }
    return ldg(a + ((size_t)k * nx + w) * nr + j);
  }
  QDS_HD void store(int field, int k, int w, int j, C<R> v) const {
#if defined(QDS_EMU)
    QDS_CHECK(gidx(field, k, w, j) < state_len, "store");
#endif
    n[gidx(field, k, w, j)] = v;
  }
  QDS_HD void store_prev(int k, int w, C<R> v) const {
    n[(size_t)NFIELD * P + (size_t)k * nx + slot(w)] = v;
  }
  QDS_HD bool owned(int lx, int lr) const {
    return lx == 0 && lr == 0 && x0 < nx && r0 < nr;
  }

  // transverse fields at time n of group grp (0 or 9), Eq. reconstruct_fields
  QDS_HD C<R> Er(int grp, int k, int w, int j) const { return R(0.5) * (cell(grp + TRP, k, w, j) + cell(grp + TRM, k, w, j)); }
  QDS_HD C<R> Bt(int grp, int k, int w, int j) const { return R(0.5) * (cell(grp + TRP, k, w, j) - cell(grp + TRM, k, w, j)); }
  QDS_HD C<R> Et(int grp, int k, int w, int j) const { return R(0.5) * (cell(grp + TTP, k, w, j) + cell(grp + TTM, k, w, j)); }
  QDS_HD C<R> Br(int grp, int k, int w, int j) const { return R(0.5) * (cell(grp + TTP, k, w, j) - cell(grp + TTM, k, w, j)); }

  // ---------------- intermediate planes ----------------
  // A plane of the new state (or scratch) at window position w;
  // out-of-domain positions read as zero and absorb writes.  Every window
  // position 0..nx-1 is a storage slot (the held-zero face nx-1 included,
  // so that it is written as zero each step).
  QDS_HD C<R> &gnew(int field, int k, int w, int j) const {
    if (FAST) {
#if defined(QDS_EMU)
      QDS_CHECK(cell_ok(w) && j >= 0 && j < nr, "unchecked new-state access");
#endif
      return n[eidx(field, k, slot(w), j)];
    }
    const bool ok = cell_ok(w) && j >= 0 && j < nr;
    if (!ok) { dummy = zero<R>(); return dummy; }
#if defined(QDS_EMU)
    QDS_CHECK(gidx(field, k, w, j) < state_len, "pass-mode new-state access");
#endif
    return n[gidx(field, k, w, j)];
  }
  QDS_HD C<R> &gscr(int plane, int k, int w, int j) const {
    if (FAST) return scr[(size_t)plane * P + ((size_t)k * nx + slot(w)) * ld + j];
    if (!cell_ok(w) || j < 0 || j >= nr) { dummy = zero<R>(); return dummy; }
    return scr[(size_t)plane * P + ((size_t)k * nx + slot(w)) * ld + j];
  }
  // lx, lr are offsets from the point (x0, r0)
  // Reads of the new state and of the scratch planes.  Each pass reads only
  // what earlier passes (earlier kernels) wrote, never what it writes
  // itself, so these reads take the non-coherent path and the compiler may
  // move them past the pass's own stores.
  QDS_HD C<R> rnew(int field, int k, int w, int j) const {
    if (FAST) {
#if defined(QDS_EMU)
      QDS_CHECK(cell_ok(w) && j >= 0 && j < nr, "unchecked new-state read");
#endif
      return ldg(n + eidx(field, k, slot(w), j));
    }
    if (!cell_ok(w) || j < 0 || j >= nr) return zero<R>();
#if defined(QDS_EMU)
    QDS_CHECK(gidx(field, k, w, j) < state_len, "pass-mode new-state read");
#endif
    return ldg(n + gidx(field, k, w, j));
  }
  QDS_HD C<R> rscr(int plane, int k, int w, int j) const {
    if (!FAST && (!cell_ok(w) || j < 0 || j >= nr)) return zero<R>();
    return ldg(scr + ((size_t)plane * P + ((size_t)k * nx + slot(w)) * ld + j));
  }
  QDS_HD C<R> rA(int pl, int k, int lx, int lr) const { return rnew(pl ? BX : EX, k, x0 + lx, r0 + lr); }
  QDS_HD C<R> rG(int k, int lx, int lr) const { return rscr(0, k, x0 + lx, r0 + lr); }
  QDS_HD C<R> rT(int pl, int k, int lx, int lr) const {
    return rnew(pl < 4 ? TRP + pl : TAP + (pl - 4), k, x0 + lx, r0 + lr);
  }
  QDS_HD C<R> rP(int k, int lx, int lr) const { return rnew(PHI, k, x0 + lx, r0 + lr); }
  QDS_HD C<R> rJ(int pl, int k, int lx, int lr) const {
    if (pl < 2) return rnew(pl ? BX1 : EX1, k, x0 + lx, r0 + lr);
    return rscr(pl - 1, k, x0 + lx, r0 + lr);
  }
  QDS_HD C<R> &sA(int pl, int k, int lx, int lr) const { return gnew(pl ? BX : EX, k, x0 + lx, r0 + lr); }  // 0: Ex0n, 1: Bx0n
  QDS_HD C<R> &sG(int k, int lx, int lr) const { return gscr(0, k, x0 + lx, r0 + lr); }
  QDS_HD C<R> &sT(int pl, int k, int lx, int lr) const {  // 0..3 T0 new, 4 Tap new, 5 Tam new
    return gnew(pl < 4 ? TRP + pl : TAP + (pl - 4), k, x0 + lx, r0 + lr);
  }
  QDS_HD C<R> &sP(int k, int lx, int lr) const { return gnew(PHI, k, x0 + lx, r0 + lr); }
  QDS_HD C<R> &sJ(int pl, int k, int lx, int lr) const {  // 0 Ex1n 1 Bx1n 2 jax 3 jar 4 jat
    if (pl < 2) return gnew(pl ? BX1 : EX1, k, x0 + lx, r0 + lr);
    return gscr(pl - 1, k, x0 + lx, r0 + lr);
  }
};

// ---------------------------------------------------------------------------
// Mode convolution C_m{A, B} (Eq. mode_convolution) for retained modes
// 0..M-1, negative modes being conjugates (Eq. fourier_decomp).
// ---------------------------------------------------------------------------
template <class R, int M>
QDS_HD C<R> conv(int m, const C<R> *A, const C<R> *B) {
  if (m == 0) {
    C<R> s = A[0] * B[0];
    R acc = R(0);
#pragma unroll
    for (int k = 1; k < M; k++) acc += A[k].re * B[k].re + A[k].im * B[k].im;
    s.re += R(0.5) * acc;
    return s;
  }
  C<R> s = zero<R>();
#pragma unroll
  for (int k = 0; k <= m && k < M; k++) {      // k + l = m
    int l = m - k;
    if (l < M) s += A[k] * B[l];
  }
#pragma unroll
  for (int l = 0; l + m < M; l++) s += mul_cj(A[l + m], B[l]);   // k - l = m
#pragma unroll
  for (int k = 0; k + m < M; k++) s += mul_cj(B[k + m], A[k]);   // l - k = m
  return R(0.5) * s;
}

// ---------------------------------------------------------------------------
// Longitudinal leapfrog (Eqs. Ex_update, Gammax_explicit, Phix_explicit,
// axis_Ex) for one mode at face w.  The radial operators are written in
// conservative form, (1/r) d(r F)/dr = (r_+ F_+ - r_- F_-)/(r dr), which is
// algebraically the paper's average-plus-centred-difference form.
// ---------------------------------------------------------------------------
template <class TT, class R = typename TT::Real>
QDS_NOINL C<R> ex_update(const TT &t, int grp, int k, int w, int j, C<R> jx) {
  C<R> e0 = t.face(grp + EX, k, w, j);
  if (j == 0) {
    if (k != 0) return zero<R>();
    C<R> b = R(0.5) * (t.Bt(grp, k, w, 0) + t.Bt(grp, k, w + 1, 0));
    return e0 + t.h * (R(4) * t.idr * b - jx);
  }
  R rj = R(j) * t.dr;
  C<R> bhi = R(0.5) * (t.Bt(grp, k, w, j) + t.Bt(grp, k, w + 1, j));
  C<R> blo = R(0.5) * (t.Bt(grp, k, w, j - 1) + t.Bt(grp, k, w + 1, j - 1));
  C<R> br = R(0.5) * (t.Br(grp, k, w, j) + t.Br(grp, k, w + 1, j));
  const R irj = R(1) / rj;  // mode-independent: the divisions stay out of the mode loops
  C<R> curl = ((R(j) + R(0.5)) * bhi - (R(j) - R(0.5)) * blo) * irj;
  C<R> gx = curl + imul(R(k) * irj, br) - jx;
  return e0 + t.h * gx;
}

template <class TT, class R = typename TT::Real>
QDS_NOINL C<R> bx_interior(const TT &t, int grp, int k, int w, int j) {
  C<R> b0 = t.face(grp + BX, k, w, j);
  R rh = (R(j) + R(0.5)) * t.dr;
  C<R> elo = R(0.5) * (t.Et(grp, k, w, j) + t.Et(grp, k, w + 1, j));
  C<R> ehi = (j + 1 < t.nr) ? R(0.5) * (t.Et(grp, k, w, j + 1) + t.Et(grp, k, w + 1, j + 1)) : zero<R>();
  C<R> er = R(0.5) * (t.Er(grp, k, w, j) + t.Er(grp, k, w + 1, j));
  const R irh = R(1) / rh;
  C<R> curl = (R(j + 1) * ehi - R(j) * elo) * irh;
  return b0 - t.h * (curl + imul(R(k) * irh, er));
}

// Outer half row J+1/2, Eq. em_r_open_bx by the box scheme over
// [r_{J-1/2}, r_{J+1/2}] x [t^{n-1/2}, t^{n+1/2}], right side at (x_{w+1/2}, r_J, t^n).
template <class TT, class R = typename TT::Real>
QDS_NOINL C<R> bx_outer(const TT &t, int grp, int k, int w, C<R> jt_face, C<R> b_in_new) {
  const int J = t.J;
  R rJ = R(J) * t.dr;
  C<R> dxbr = t.ih * (t.Br(grp, k, w + 1, J) - t.Br(grp, k, w, J));
  C<R> eth = R(0.5) * (t.Et(grp, k, w, J) + t.Et(grp, k, w + 1, J));
  C<R> er = R(0.25) * (t.Er(grp, k, w, J - 1) + t.Er(grp, k, w, J) + t.Er(grp, k, w + 1, J - 1) + t.Er(grp, k, w + 1, J));
  C<R> rhs = R(0.5) * dxbr - (R(0.5) / rJ) * (eth + imul(R(k), er)) - R(0.5) * jt_face;
  C<R> bo = t.face(grp + BX, k, w, J), bi = t.face(grp + BX, k, w, J - 1);
  R a = R(0.5) * t.ih, b = R(0.5) * t.idr;
  C<R> num = rhs - (a - b) * b_in_new + (a - b) * bo + (a + b) * bi;
  return num * (R(1) / (a + b));
}

// Both longitudinal updates of one mode at face w, with each transverse
// value loaded once: E_x from B_theta on half rows j-1, j and B_r on row j;
// B_x from E_theta on rows j, j+1 and E_r on half row j (the same
// expressions as ex_update and bx_interior; the outer row takes bx_outer).
template <class TT, class R = typename TT::Real>
QDS_NOINL void leap_point(const TT &t, int grp, int k, int w, int j, C<R> jx, C<R> jt_face,
                          C<R> &ex, C<R> &bx) {
  // cell sums over w, w+1 of the reconstructed fields (Eq. reconstruct_fields)
  const C<R> rp = t.cell(grp + TRP, k, w, j) + t.cell(grp + TRP, k, w + 1, j);
  const C<R> rm = t.cell(grp + TRM, k, w, j) + t.cell(grp + TRM, k, w + 1, j);
  const C<R> qp = t.cell(grp + TTP, k, w, j) + t.cell(grp + TTP, k, w + 1, j);
  const C<R> qm = t.cell(grp + TTM, k, w, j) + t.cell(grp + TTM, k, w + 1, j);
  const C<R> er = R(0.25) * (rp + rm), bth = R(0.25) * (rp - rm);
  const C<R> eth = R(0.25) * (qp + qm), brr = R(0.25) * (qp - qm);
  const C<R> e0 = t.face(grp + EX, k, w, j);
  if (j == 0) {
    ex = (k != 0) ? zero<R>() : e0 + t.h * (R(4) * t.idr * bth - jx);
  } else {
    const C<R> rpl = t.cell(grp + TRP, k, w, j - 1) + t.cell(grp + TRP, k, w + 1, j - 1);
    const C<R> rml = t.cell(grp + TRM, k, w, j - 1) + t.cell(grp + TRM, k, w + 1, j - 1);
    const C<R> blo = R(0.25) * (rpl - rml);
    const R irj = R(1) / (R(j) * t.dr);
    const C<R> curl = ((R(j) + R(0.5)) * bth - (R(j) - R(0.5)) * blo) * irj;
    ex = e0 + t.h * (curl + imul(R(k) * irj, brr) - jx);
  }
  if (j == t.J && !t.closed) {
    bx = bx_outer(t, grp, k, w, jt_face, bx_interior(t, grp, k, w, j - 1));
    return;
  }
  C<R> ehi = zero<R>();
  if (j + 1 < t.nr) {
    const C<R> qp1 = t.cell(grp + TTP, k, w, j + 1) + t.cell(grp + TTP, k, w + 1, j + 1);
    const C<R> qm1 = t.cell(grp + TTM, k, w, j + 1) + t.cell(grp + TTM, k, w + 1, j + 1);
    ehi = R(0.25) * (qp1 + qm1);
  }
  const R irh = R(1) / ((R(j) + R(0.5)) * t.dr);
  const C<R> curl = (R(j + 1) * ehi - R(j) * eth) * irh;
  bx = t.face(grp + BX, k, w, j) - t.h * (curl + imul(R(k) * irh, er));
}

// ---------------------------------------------------------------------------
// Face quantities consumed by the characteristic shift: group 0 reads them
// from the tile's shared memory and x-averages the caller's cell currents;
// group 1 (the regenerated field) reads E_x1, B_x1 and j_a from shared memory.
// ---------------------------------------------------------------------------
template <class TT>
struct Faces0 {
  using R = typename TT::Real;
  const TT &t;
  QDS_HD C<R> ex(int k, int lx, int lr) const { return t.rA(0, k, lx, lr); }
  QDS_HD C<R> bx(int k, int lx, int lr) const { return t.rA(1, k, lx, lr); }
  QDS_HD C<R> jr(int k, int lx, int lr) const {
    int w = t.x0 + lx, j = t.r0 + lr;
    if (!t.jr || !t.face_ok(w)) return zero<R>();
    return R(0.5) * (t.srcv(t.jr, k, w, j) + t.srcv(t.jr, k, w + 1, j));
  }
  QDS_HD C<R> jt(int k, int lx, int lr) const {
    int w = t.x0 + lx, j = t.r0 + lr;
    if (!t.jt || !t.face_ok(w)) return zero<R>();
    return R(0.5) * (t.srcv(t.jt, k, w, j) + t.srcv(t.jt, k, w + 1, j));
  }
  QDS_HD C<R> jx(int k, int lx, int lr) const {
    int w = t.x0 + lx, j = t.r0 + lr;
    if (!t.face_ok(w)) return zero<R>();
    return t.srcv(t.jx, k, w, j);
  }
};

template <class TT>
struct Faces1 {
  using R = typename TT::Real;
  const TT &t;
  QDS_HD C<R> ex(int k, int lx, int lr) const { return t.rJ(0, k, lx, lr); }
  QDS_HD C<R> bx(int k, int lx, int lr) const { return t.rJ(1, k, lx, lr); }
  QDS_HD C<R> jx(int k, int lx, int lr) const { return t.rJ(2, k, lx, lr); }
  QDS_HD C<R> jr(int k, int lx, int lr) const { return t.rJ(3, k, lx, lr); }
  QDS_HD C<R> jt(int k, int lx, int lr) const { return t.rJ(4, k, lx, lr); }
};

// ---------------------------------------------------------------------------
// Characteristic shift of the transport variables (Eqs. Trp_update,
// Trm_update, Ttp_update, Ttm_update): T_r^+ and T_th^- arrive from the cell
// behind through face c-1, T_r^- and T_th^+ from the cell ahead through face
// c.  Axis rules of Sec. 2.3 (Eq. axis_Ttheta; T_th^(m!=1) = 0 on the axis).
// ---------------------------------------------------------------------------
template <class TT, class FS, class R = typename TT::Real>
QDS_NOINL void tr_interior(const TT &t, const FS &fs, int grp, int k, int lx, int lr, C<R> &tp, C<R> &tm) {
  const int c = t.x0 + lx, j = t.r0 + lr;
  const R irh = R(1) / ((R(j) + R(0.5)) * t.dr);
  C<R> sp = zero<R>(), sm = zero<R>();
  if (t.face_ok(c - 1)) {
    C<R> ehi = (j + 1 < t.nr) ? fs.ex(k, lx - 1, lr + 1) : zero<R>();
    C<R> gr = -imul(R(k) * irh, fs.bx(k, lx - 1, lr)) - fs.jr(k, lx - 1, lr);
    sp = gr + t.idr * (ehi - fs.ex(k, lx - 1, lr));
  }
  if (t.face_ok(c)) {
    C<R> ehi = (j + 1 < t.nr) ? fs.ex(k, lx, lr + 1) : zero<R>();
    C<R> gr = -imul(R(k) * irh, fs.bx(k, lx, lr)) - fs.jr(k, lx, lr);
    sm = gr - t.idr * (ehi - fs.ex(k, lx, lr));
  }
  tp = t.cell(grp + TRP, k, c - 1, j) + t.h * sp;
  tm = t.cell(grp + TRM, k, c + 1, j) + t.h * sm;
}

// Outer half row: E_r by the shift with the Gamma_r source alone, B_theta by
// the box scheme of Eq. em_r_open_bt over [r_{J-1/2}, r_{J+1/2}] x [t^n, t^{n+1}]
// with its right side from time-n fields.
template <class TT, class FS, class R = typename TT::Real>
QDS_NOINL void tr_outer(const TT &t, const FS &fs, int grp, int k, int lx, C<R> bt_in_new, int lr_J, C<R> &tp,
                        C<R> &tm) {
  const int c = t.x0 + lx, J = t.J;
  const R irh = R(1) / ((R(J) + R(0.5)) * t.dr), rJ = R(J) * t.dr;
  C<R> gl = zero<R>(), gr = zero<R>();
  if (t.face_ok(c - 1)) gl = -imul(R(k) * irh, fs.bx(k, lx - 1, lr_J)) - fs.jr(k, lx - 1, lr_J);
  if (t.face_ok(c)) gr = -imul(R(k) * irh, fs.bx(k, lx, lr_J)) - fs.jr(k, lx, lr_J);
  C<R> er_new = R(0.5) * (t.cell(grp + TRP, k, c - 1, J) + t.cell(grp + TRM, k, c + 1, J) + t.h * (gl + gr));
  C<R> erl = R(0.5) * (t.Er(grp, k, c - 1, J - 1) + t.Er(grp, k, c - 1, J));
  C<R> err = R(0.5) * (t.Er(grp, k, c + 1, J - 1) + t.Er(grp, k, c + 1, J));
  C<R> bth = R(0.5) * (t.Bt(grp, k, c, J - 1) + t.Bt(grp, k, c, J));
  C<R> br = t.Br(grp, k, c, J);
  C<R> jxl = t.face_ok(c - 1) ? fs.jx(k, lx - 1, lr_J) : zero<R>();
  C<R> jxr = t.face_ok(c) ? fs.jx(k, lx, lr_J) : zero<R>();
  C<R> rhs = (R(-0.25) * t.ih) * (err - erl) - (R(0.5) / rJ) * (bth + imul(R(k), br)) + R(0.25) * (jxl + jxr);
  C<R> bo = t.Bt(grp, k, c, J), bi = t.Bt(grp, k, c, J - 1);
  R a = R(0.5) * t.ih, b = R(0.5) * t.idr;
  C<R> bt_new = (rhs - (a - b) * bt_in_new + (a - b) * bo + (a + b) * bi) * (R(1) / (a + b));
  tp = er_new + bt_new;
  tm = er_new - bt_new;
}

template <class TT, class FS, class R = typename TT::Real>
QDS_NOINL void tt_update(const TT &t, const FS &fs, int grp, int k, int lx, int lr, C<R> &tp, C<R> &tm) {
  const int c = t.x0 + lx, j = t.r0 + lr;
  if (j == 0 && k != 1) { tp = zero<R>(); tm = zero<R>(); return; }
  C<R> sp = zero<R>(), sm = zero<R>();
  for (int side = 0; side < 2; side++) {
    const int lf = side == 0 ? lx : lx - 1;  // + from face c, - from face c-1
    if (!t.face_ok(t.x0 + lf)) continue;
    C<R> g, p;
    if (j == 0) {
      g = -(R(2) * t.idr) * fs.bx(k, lf, lr) - fs.jt(k, lf, lr);
      p = imul(t.idr, fs.ex(k, lf, lr + 1) - fs.ex(k, lf, lr));
    } else {
      g = -t.idr * (fs.bx(k, lf, lr) - fs.bx(k, lf, lr - 1)) - fs.jt(k, lf, lr);
      p = imul(R(k) * (R(1) / (R(j) * t.dr)), fs.ex(k, lf, lr));
    }
    if (side == 0) sp = g + p; else sm = g - p;
  }
  tp = t.cell(grp + TTP, k, c + 1, j) + t.h * sp;
  tm = t.cell(grp + TTM, k, c - 1, j) + t.h * sm;
}


// ---------------------------------------------------------------------------
// Axion source and Klein-Gordon operator at face w, half row j, time n:
//   S_a^(m) = sum_alpha C_m{E_alpha, B_alpha}  (Eqs. source_mode_zero/_m),
//   Gamma_a = (1/r) d/dr (r dphi/dr) - m^2 phi / r^2 - m_a^2 phi + g S_a.
// Every field component is averaged onto (x_{w+1/2}, r_{j+1/2}); E_x and B_x
// also over the levels n -+ 1/2.  Beyond the outermost half row the
// exterior phi comes from the outgoing condition (d_t + c d_r) phi = 0
// centred at r_J (Eq. axion_r_ghost) with d_t phi taken half a step back.
// ---------------------------------------------------------------------------
// Provider of E_x^(n+1/2), B_x^(n+1/2) at face x0+lx (rows lr, lr+1): the
// accessor's intermediate planes.
template <class TT>
struct TileLeapVals {
  using R = typename TT::Real;
  const TT &t;
  int lx, lr;
  QDS_HD C<R> exn(int k, int dj) const { return t.rA(0, k, lx, lr + dj); }
  QDS_HD C<R> bxn(int k) const { return t.rA(1, k, lx, lr); }
};

// m_only >= 0: only the output mode m_only (the inputs of all modes are
// still formed), so that the modes of a point can be spread over threads.
template <class TT, class NV>
QDS_NOINL void source_point(const TT &t, int lx, int lr, const NV &nv, int m_only = -1) {
  using R = typename TT::Real;
  constexpr int M = TT::kM;
  const int w = t.x0 + lx, j = t.r0 + lr;
  if (!t.face_ok(w) || j < 0 || j >= t.nr) {
    for (int k = 0; k < M; k++)
      if (m_only < 0 || k == m_only) t.sG(k, lx, lr) = zero<R>();
    return;
  }
  const bool top = (j == t.J);
  // E_x B_x term, and the transverse term written in transport variables:
  // with E_r, B_theta from the same x-average of T_r and E_theta, B_r from
  // the same four-point average of T_theta, the symmetry of C_m gives
  //   C{E_r, B_r} + C{E_th, B_th} = (1/2)(C{Tr+, Tth+} - C{Tr-, Tth-}),
  // free of the cancellation of E.B between co-propagating waves (Eq.
  // mixing_source: zero in vacuum).
  C<R> eX[M], bX[M], rp[M], rm[M], qp[M], qm[M];
#pragma unroll
  for (int k = 0; k < M; k++) {
    C<R> eo = t.face(EX, k, w, j), en = nv.exn(k, 0), eo1, en1;
    if (!top) { eo1 = t.face(EX, k, w, j + 1); en1 = nv.exn(k, 1); }
    else if (t.closed) { eo1 = zero<R>(); en1 = zero<R>(); }
    else { eo1 = eo; en1 = en; }
    eX[k] = R(0.25) * (eo + eo1 + en + en1);
    bX[k] = R(0.5) * (t.face(BX, k, w, j) + nv.bxn(k));
    rp[k] = R(0.5) * (t.cell(TRP, k, w, j) + t.cell(TRP, k, w + 1, j));
    rm[k] = R(0.5) * (t.cell(TRM, k, w, j) + t.cell(TRM, k, w + 1, j));
    C<R> p0 = t.cell(TTP, k, w, j) + t.cell(TTP, k, w + 1, j);
    C<R> m0 = t.cell(TTM, k, w, j) + t.cell(TTM, k, w + 1, j);
    C<R> p1, m1;
    if (!top) { p1 = t.cell(TTP, k, w, j + 1) + t.cell(TTP, k, w + 1, j + 1); m1 = t.cell(TTM, k, w, j + 1) + t.cell(TTM, k, w + 1, j + 1); }
    else if (t.closed) { p1 = zero<R>(); m1 = zero<R>(); }
    else { p1 = p0; m1 = m0; }
    qp[k] = R(0.25) * (p0 + p1);
    qm[k] = R(0.25) * (m0 + m1);
  }
  const R idr2 = t.idr * t.idr;
  const R rh = (R(j) + R(0.5)) * t.dr;
  const R irh2 = R(1) / (rh * rh);
#pragma unroll
  for (int m = 0; m < M; m++) {
    if (m_only >= 0 && m != m_only) continue;
    C<R> S = conv<R, M>(m, eX, bX) + R(0.5) * (conv<R, M>(m, rp, qp) - conv<R, M>(m, rm, qm));
    S += t.srcv(t.sext, m, w, j);
    C<R> pc = t.face(PHI, m, w, j);
    C<R> pm = (j > 0) ? t.face(PHI, m, w, j - 1) : zero<R>();  // weight j = 0 on the axis
    C<R> pp;
    if (!top) pp = t.face(PHI, m, w, j + 1);
    else if (t.closed) pp = pc;
    else pp = t.face(PHI, m, w, j - 1) - (R(2) * t.dr * t.ih) * (pc - t.prev(m, w));
    C<R> lap = (R(j + 1) * (pp - pc) - R(j) * (pc - pm)) * (idr2 / (R(j) + R(0.5)));
    C<R> ga = lap - (R(m * m) * irh2 + t.ma2) * pc + t.gs * S;
    t.sG(m, lx, lr) = ga;
  }
}

template <class TT>
QDS_NOINL void source_point(const TT &t, int lx, int lr) {
  source_point(t, lx, lr, TileLeapVals<TT>{t, lx, lr});
}

// ---------------------------------------------------------------------------
// Axion current j_a = g (B0 d_t phi - E0 x grad phi) (Eqs. jax_mode,
// jar_mode, jat_mode), with (d_theta phi)^(l) = -i l phi^(l):
//   j_a,x at (x_{w+1/2}, r_j, t^n), j_a,r at (x_{w+1/2}, r_{j+1/2}, t^{n+1/2}),
//   j_a,theta at (x_{w+1/2}, r_j, t^{n+1/2}).
// d_t phi = (c/2)(T_a^+ + T_a^-), d_x phi = (1/2)(T_a^- - T_a^+) (Eq. phi_update).
// Below the axis a scalar on half rows mirrors with parity (-1)^l; E_r and
// B_theta below the axis follow the T_r ghost of Eq. axis_Tr.
// ---------------------------------------------------------------------------
// Provider of the values of the new level that j_a needs around face
// x0+lx: ns(pl, k, jj) = sum over cells x0+lx, x0+lx+1 of plane pl (0..3:
// T_r^+, T_r^-, T_th^+, T_th^- at n+1; 4, 5: T_a^+, T_a^- at n+1/2) on row
// jj, and pn(k, jj) = phi^(n+1) at the face on row jj.
template <class TT>
struct TileNewVals {
  using R = typename TT::Real;
  const TT &t;
  int lx;
  QDS_HD C<R> ns(int pl, int k, int jj) const {
    const int l = jj - t.r0;
    return t.rT(pl, k, lx, l) + t.rT(pl, k, lx + 1, l);
  }
  QDS_HD C<R> pn(int k, int jj) const { return t.rP(k, lx, jj - t.r0); }
};

// comp selects the components computed (bit 0: j_a,x, 1: j_a,r, 2:
// j_a,theta), so that they can be spread over threads.
template <class TT, class NV, class R = typename TT::Real, int M = TT::kM>
QDS_NOINL void current_point(const TT &t, int lx, int lr, C<R> (&jax)[M], C<R> (&jat)[M], const NV &nv,
                             int comp = 7) {
  constexpr bool SM = TT::kSM;
  const int w = t.x0 + lx, j = t.r0 + lr;
  if (!t.face_ok(w) || j < 0 || j >= t.nr) {
    for (int k = 0; k < M; k++) {
      for (int q = 2; q < 5; q++)
        if ((comp >> (q - 2)) & 1)
          if (SM || q > 2 || j == t.J) t.sJ(q, k, lx, lr) = zero<R>();
      jax[k] = jat[k] = zero<R>();
    }
    return;
  }
  const bool top = (j == t.J);
  const int j1 = top ? -1 : j + 1;  // row above, -1: beyond the last row
  const R gj = t.gj;
  const R ih = t.ih;
  // ---- j_a,x at (w, j, n) ----
  if (comp & 1) {
    C<R> a1[M], b1[M], a2[M], b2[M], a3[M], b3[M];
#pragma unroll
    for (int k = 0; k < M; k++) {
      const R par = (k & 1) ? R(-1) : R(1);
      C<R> bx_hi = R(0.5) * (t.face(BX, k, w, j) + t.rA(1, k, lx, lr));
      C<R> bx_lo = (j > 0) ? R(0.5) * (t.face(BX, k, w, j - 1) + t.rA(1, k, lx, lr - 1)) : par * bx_hi;
      a1[k] = R(0.5) * (bx_lo + bx_hi);
      C<R> dt_hi = R(0.125) * (t.cell(TAP, k, w, j) + t.cell(TAM, k, w, j) + t.cell(TAP, k, w + 1, j) + t.cell(TAM, k, w + 1, j) +
                               nv.ns(4, k, j) + nv.ns(5, k, j));
      C<R> dt_lo;
      if (j > 0)
        dt_lo = R(0.125) * (t.cell(TAP, k, w, j - 1) + t.cell(TAM, k, w, j - 1) + t.cell(TAP, k, w + 1, j - 1) + t.cell(TAM, k, w + 1, j - 1) +
                            nv.ns(4, k, j - 1) + nv.ns(5, k, j - 1));
      else dt_lo = par * dt_hi;
      b1[k] = R(0.5) * (dt_lo + dt_hi);
      C<R> er_hi = R(0.5) * (t.Er(0, k, w, j) + t.Er(0, k, w + 1, j)), er_lo;
      if (j > 0) er_lo = R(0.5) * (t.Er(0, k, w, j - 1) + t.Er(0, k, w + 1, j - 1));
      else if (k == 1) er_lo = imul(R(1), t.Et(0, k, w, 0) + t.Et(0, k, w + 1, 0)) - er_hi;
      else er_lo = -er_hi;
      a2[k] = R(0.5) * (er_lo + er_hi);
      C<R> ph = t.face(PHI, k, w, j);
      C<R> pl = (j > 0) ? t.face(PHI, k, w, j - 1) : par * ph;
      if (j > 0) b2[k] = imul(-R(k) * R(0.5) * (R(1) / (R(j) * t.dr)), pl + ph);
      else b2[k] = (k == 1) ? imul(-t.idr, ph - pl) : zero<R>();
      a3[k] = R(0.5) * (t.Et(0, k, w, j) + t.Et(0, k, w + 1, j));
      b3[k] = t.idr * (ph - pl);
    }
#pragma unroll
    for (int m = 0; m < M; m++) {
      jax[m] = gj * (conv<R, M>(m, a1, b1) - conv<R, M>(m, a2, b2) + conv<R, M>(m, a3, b3));
      // pass mode: consumed by the caller, and on the outer row by the
      // box scheme of the regenerated shift
      if (SM || j == t.J) t.sJ(2, m, lx, lr) = jax[m];
    }
  }
  // Transport variables at time n + 1/2 (mean of level n, global, and
  // level n+1, the new state), summed over cells w and w+1.  With E, B at
  // n + 1/2 from these means, E_th + B_r = T_th^+ and E_th - B_r = T_th^-,
  // E_r + B_th = T_r^+ and E_r - B_th = T_r^-, so the sums below are the
  // cell sums of those combinations.
  auto QP = [&](int k, int jj) -> C<R> {  // T_th^+ on row jj
    return R(0.5) * (t.cell(TTP, k, w, jj) + t.cell(TTP, k, w + 1, jj) + nv.ns(2, k, jj));
  };
  auto QM = [&](int k, int jj) -> C<R> {  // T_th^- on row jj
    return R(0.5) * (t.cell(TTM, k, w, jj) + t.cell(TTM, k, w + 1, jj) + nv.ns(3, k, jj));
  };
  auto RP = [&](int k, int jj) -> C<R> {  // T_r^+ on half row jj
    return R(0.5) * (t.cell(TRP, k, w, jj) + t.cell(TRP, k, w + 1, jj) + nv.ns(0, k, jj));
  };
  auto RM = [&](int k, int jj) -> C<R> {  // T_r^- on half row jj
    return R(0.5) * (t.cell(TRM, k, w, jj) + t.cell(TRM, k, w + 1, jj) + nv.ns(1, k, jj));
  };

  // Mean over cells w, w+1 of T_a^+- at n+1/2 on half row jj (the new
  // level, shared memory).  In the scheme (phi^(n+1) - phi^n)/dt equals
  // (1/2)(Ta+ + Ta-) of this mean on every half row (Eq. phi_update), and
  // d_x phi = (1/2)(Ta- - Ta+).
  auto TAX = [&](int pl, int k, int jj) -> C<R> {  // pl 4: Ta+, 5: Ta-
    return R(0.5) * nv.ns(pl, k, jj);
  };
  // ---- j_a,r at (w, j + 1/2, n + 1/2) ----
  //   C{B_r, d_t phi} - C{E_th, d_x phi} = (1/2)(C{Tth+, Ta+} - C{Tth-, Ta-})
  // with T_theta averaged over cells w, w+1, rows j, j+1 and levels n, n+1.
  if (comp & 2) {
    C<R> a1[M], b1[M], a2[M], b2[M], a3[M], b3[M];
#pragma unroll
    for (int k = 0; k < M; k++) {
      C<R> p = QP(k, j);   // Tth+ summed over cells w, w+1
      C<R> m = QM(k, j);
      C<R> p1, m1;
      if (j1 >= 0) {
        p1 = QP(k, j1);
        m1 = QM(k, j1);
      } else if (t.closed) { p1 = zero<R>(); m1 = zero<R>(); }
      else { p1 = p; m1 = m; }
      a1[k] = R(0.25) * (p + p1);
      a2[k] = R(0.25) * (m + m1);
      b1[k] = TAX(4, k, j);
      b2[k] = TAX(5, k, j);
      C<R> po = t.face(PHI, k, w, j), pn = nv.pn(k, j);
      C<R> ex_lo = t.rA(0, k, lx, lr), ex_hi;
      if (j1 >= 0) ex_hi = t.rA(0, k, lx, lr + 1);
      else ex_hi = t.closed ? zero<R>() : ex_lo;
      a3[k] = R(0.5) * (ex_lo + ex_hi);
      b3[k] = imul(-R(k) * R(0.5) * (R(1) / ((R(j) + R(0.5)) * t.dr)), po + pn);
    }
#pragma unroll
    for (int m = 0; m < M; m++)
      t.sJ(3, m, lx, lr) = gj * (R(0.5) * (conv<R, M>(m, a1, b1) - conv<R, M>(m, a2, b2)) + conv<R, M>(m, a3, b3));
  }
  // ---- j_a,theta at (w, j, n + 1/2) ----
  //   C{B_th, d_t phi} + C{E_r, d_x phi} = (1/2)(C{Tr+, Ta-} - C{Tr-, Ta+})
  // with T_r averaged over cells w, w+1, half rows j -+ 1/2 and levels n,
  // n+1; below the axis T_r^+-(-1/2) = 2i T_th^-+(0) - T_r^+-(1/2) (m = 1,
  // Eq. axis_Tr) and -T_r(1/2) otherwise, so on the axis the average is
  // i T_th^-+(0) for m = 1 and zero otherwise.
  if (comp & 4) {
    C<R> a1[M], b1[M], a2[M], b2[M], a3[M], b3[M];
#pragma unroll
    for (int k = 0; k < M; k++) {
      const R par = (k & 1) ? R(-1) : R(1);
      if (j > 0) {
        a1[k] = R(0.25) * (RP(k, j) + RP(k, j - 1));
        a2[k] = R(0.25) * (RM(k, j) + RM(k, j - 1));
      } else if (k == 1) {
        C<R> tm0 = R(0.5) * QM(k, 0);  // Tth- at the axis
        C<R> tp0 = R(0.5) * QP(k, 0);  // Tth+
        a1[k] = imul(R(1), tm0);
        a2[k] = imul(R(1), tp0);
      } else {
        a1[k] = zero<R>();
        a2[k] = zero<R>();
      }
      C<R> ap_hi = TAX(4, k, j), am_hi = TAX(5, k, j);
      C<R> ap_lo = (j > 0) ? TAX(4, k, j - 1) : par * ap_hi;
      C<R> am_lo = (j > 0) ? TAX(5, k, j - 1) : par * am_hi;
      b1[k] = R(0.5) * (am_lo + am_hi);   // Ta- paired with Tr+
      b2[k] = R(0.5) * (ap_lo + ap_hi);   // Ta+ paired with Tr-
      a3[k] = t.rA(0, k, lx, lr);
      C<R> pbh = R(0.5) * (t.face(PHI, k, w, j) + nv.pn(k, j));
      C<R> pbl = (j > 0) ? R(0.5) * (t.face(PHI, k, w, j - 1) + nv.pn(k, j - 1)) : par * pbh;
      b3[k] = t.idr * (pbh - pbl);
    }
#pragma unroll
    for (int m = 0; m < M; m++) {
      jat[m] = gj * (R(0.5) * (conv<R, M>(m, a1, b1) - conv<R, M>(m, a2, b2)) - conv<R, M>(m, a3, b3));
      t.sJ(4, m, lx, lr) = jat[m];
    }
  }
}

template <class TT, class R = typename TT::Real, int M = TT::kM>
QDS_NOINL void current_point(const TT &t, int lx, int lr, C<R> (&jax)[M], C<R> (&jat)[M]) {
  current_point(t, lx, lr, jax, jat, TileNewVals<TT>{t, lx});
}

// ---------------------------------------------------------------------------
// Pass-mode stages over single points (x0, r0) of the grid, one point per
// thread with all modes; each stage is its own kernel (qds_kernels.cuh):
//   ST_LEAP0    E_x, B_x to n+1/2 (into the new state)
//   ST_SOURCE   Gamma_a at n (scratch plane 0)
//   ST_SHIFT0   T, T_a to n+1 / n+1/2 and phi to n+1 (phi of face c is formed
//               from T_a^(n+1/2) of cells c and c+1, the latter rebuilt here
//               from Gamma_a of faces c, c+1)
//   ST_CURRENT  j_a (scratch planes 1..3) and the regenerated leapfrog
//   ST_SHIFT1   the regenerated shift
//   ST_ZERO     moving window: the rear column of every field becomes the new
//               (empty) front column once all passes have read it
// ---------------------------------------------------------------------------
enum Stage { ST_LEAP0 = 0, ST_SOURCE, ST_SHIFT0, ST_CURRENT, ST_SHIFT1, ST_ZERO, N_STAGE };

template <class R, int M, bool FAST = false>
QDS_HD void run_stage(Tile<R, M, FAST> t, int st) {
  const uint32_t fl = t.flags;
  const bool ax = (fl & (F_AXION | F_AREM)) != 0, ar = (fl & F_AREM) != 0;
  const int lx = 0, lr = 0;
  if (!t.owned(lx, lr)) return;
  if (st == ST_ZERO) {
    if (!t.mw || t.x0 != 0) return;
    t.set_point(0);
    const int j = t.r0;
    for (int f = 0; f < NFIELD; f++)
      for (int k = 0; k < M; k++) t.n[t.gidx(f, k, 0, j)] = zero<R>();
    if (j == t.J)
      for (int k = 0; k < M; k++) t.n[(size_t)NFIELD * t.P + (size_t)k * t.nx + t.slot(0)] = zero<R>();
    return;
  }
  if (st == ST_LEAP0) {
    const int w = t.x0, j = t.r0;
    t.set_point(w);
    const bool live = t.face_ok(w) && j >= 0 && j < t.nr;
#pragma unroll 1
    for (int k = 0; k < M; k++) {
      C<R> ex = zero<R>(), bx = zero<R>();
      if (live) {
        C<R> jtf = zero<R>();
        if (j == t.J && !t.closed) jtf = R(0.5) * (t.srcv(t.jt, k, w, j) + t.srcv(t.jt, k, w + 1, j));
        leap_point(t, 0, k, w, j, t.srcv(t.jx, k, w, j), jtf, ex, bx);
      }
      t.sA(0, k, lx, lr) = ex;
      t.sA(1, k, lx, lr) = bx;
    }
  } else if (st == ST_SOURCE) {
    if (!ax) return;
    t.set_point(t.x0);
    source_point(t, lx, lr);
  } else if (st == ST_SHIFT0) {
    Faces0<Tile<R, M, FAST>> fs{t};
    const int c = t.x0, j = t.r0;
    t.set_point(c);  // the shift reads cells c-1 .. c+1 (phi: c+2)
    const bool live = t.cell_ok(c) && j >= 0 && j < t.nr;
#pragma unroll 1
    for (int k = 0; k < M; k++) {
      C<R> tp = zero<R>(), tm = zero<R>(), up = zero<R>(), um = zero<R>();
      C<R> ap = zero<R>(), am = zero<R>();
      if (live) {
        if (j < t.J || t.closed) tr_interior(t, fs, 0, k, lx, lr, tp, tm);
        else {
          C<R> ip, im_;
          tr_interior(t, fs, 0, k, lx, lr - 1, ip, im_);
          tr_outer(t, fs, 0, k, lx, R(0.5) * (ip - im_), lr, tp, tm);
        }
        tt_update(t, fs, 0, k, lx, lr, up, um);
        if (ax) {
          ap = t.cell(TAP, k, c - 1, j) + t.h * t.rG(k, lx - 1, lr);
          am = t.cell(TAM, k, c + 1, j) + t.h * t.rG(k, lx, lr);
        }
      }
      t.store(TRP, k, c, j, tp); t.store(TRM, k, c, j, tm);
      t.store(TTP, k, c, j, up); t.store(TTM, k, c, j, um);
      if (ax) {
        t.store(TAP, k, c, j, ap); t.store(TAM, k, c, j, am);
        // phi at face c (Eq. phi_update) from T_a^(n+1/2) of cells c (above)
        // and c+1 (formed here from Gamma_a of faces c, c+1)
        const bool flive = t.face_ok(c) && j >= 0 && j < t.nr;
        C<R> v = zero<R>(), po = zero<R>();
        if (flive) {
          const C<R> ap1 = t.cell(TAP, k, c, j) + t.h * t.rG(k, lx, lr);
          const C<R> am1 = t.cell(TAM, k, c + 2, j) + t.h * t.rG(k, lx + 1, lr);
          po = t.face(PHI, k, c, j);
          v = po + (R(0.25) * t.h) * (am1 + am + ap1 + ap);
        }
        t.sP(k, lx, lr) = v;
        if (j == t.J) t.store_prev(k, c, po);
      }
    }
  } else if (st == ST_CURRENT) {
    if (!ar) return;
    const int w = t.x0, j = t.r0;
    t.set_point(w);
    C<R> jax[M], jat[M];
    current_point(t, lx, lr, jax, jat, TileNewVals<Tile<R, M, FAST>>{t, lx});
    // the regenerated leapfrog (Sec. 2.2) of this face follows at once; it
    // needs j_a,x and (outer row) j_a,theta of this point only
    const bool live = t.face_ok(w) && j >= 0 && j < t.nr;
#pragma unroll 1
    for (int k = 0; k < M; k++) {
      C<R> ex = zero<R>(), bx = zero<R>();
      if (live) leap_point(t, 9, k, w, j, jax[k], jat[k], ex, bx);
      t.sJ(0, k, lx, lr) = ex;
      t.sJ(1, k, lx, lr) = bx;
    }
  } else if (st == ST_SHIFT1) {
    if (!ar) return;
    Faces1<Tile<R, M, FAST>> fs{t};
    const int c = t.x0, j = t.r0;
    t.set_point(c);
#pragma unroll 1
    for (int k = 0; k < M; k++) {
      C<R> tp, tm, up, um;
      if (j < t.J || t.closed) tr_interior(t, fs, 9, k, lx, lr, tp, tm);
      else {
        C<R> ip, im_;
        tr_interior(t, fs, 9, k, lx, lr - 1, ip, im_);
        tr_outer(t, fs, 9, k, lx, R(0.5) * (ip - im_), lr, tp, tm);
      }
      tt_update(t, fs, 9, k, lx, lr, up, um);
      t.store(TRP1, k, c, j, tp); t.store(TRM1, k, c, j, tm);
      t.store(TTP1, k, c, j, up); t.store(TTM1, k, c, j, um);
    }
  }
}

}  // namespace qds
