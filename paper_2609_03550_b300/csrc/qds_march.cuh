// qds_march.cuh -- the x-marching step kernels.
//
// One CTA owns a band of radial rows [r0, r1) of one instance, all retained
// modes, and a segment of window columns [xa, xb); it walks the segment along
// +x one column per iteration.  Each column of the old state (nine planes,
// all modes, the band and its radial halo) arrives in a ring of shared-memory
// slots by one bulk tensor copy (TMA) completed on an mbarrier, two columns
// ahead of the column being computed.  Columns outside the window and rows
// outside the grid come in as zeros from the copy's out-of-range fill, which
// is the open boundary of Eqs. em_x_open / axion_x_open; the moving window is
// the copy's column coordinate (the ring offset), not a data move.
//
// Thread (k, lr) of a CTA owns mode k and ring row lr (row j = rb0 + lr); a
// warp is 32 consecutive rows of one mode, so every shared-memory access of a
// plane is 32 consecutive 8-byte (FP32) words.  The radius factors of the
// thread's row and mode are formed once.  Two kernels per step:
//
// K1 (EM field, axion, axion current), iteration L (column L has landed):
//   P1  A   E_x, B_x to n+1/2 at face L-1 (Eqs. Ex_update, Phix_explicit,
//           axis_Ex, em_r_open_bx); keeps the face quantities the axion
//           source and current need (cell sums of the old T, B_x at n)
//   P2  per row, one task per thread of the row's mode threads:
//           S    S_a of every mode at face L-1 (Eqs. source_mode_*,
//                mode_convolution)
//           Dx, Dr, Dth  j_a of every mode at face L-3 (Eqs. jax/jar/jat_mode)
//   P3  Gamma_a at face L-1 (Eq. axion_waveeq discretised), the shift of
//       T and T_a at cell L-1 (Eqs. Trp..Ttm_update, Ta_plus/minus_update,
//       axis_Ttheta, em_r_open_bt), phi at face L-2 (Eq. phi_update)
// K2 (axion-regenerated EM field driven by j_a, Sec. 2.2):
//   P1  A'  E_x1, B_x1 at face L-1;   P2  C'  T1 at cell L-2.
// A barrier separates the phases.  The state is read once and written once
// per step (K1: 9 planes and the 3 j_a planes written; K2: 6 planes and the
// 3 j_a planes read back).
#pragma once

#include "qds_stages.cuh"

#if defined(__CUDACC__) && !defined(QDS_EMU)
#include <cuda.h>

#include "qds_kernels.cuh"
#endif

// Rarely taken boundary code (the outer half row) is kept out of line on the
// device, so that the hot loop body stays small in the instruction cache.
#if defined(__CUDACC__) && !defined(QDS_EMU)
#define QDS_COLD __device__ __noinline__
#else
#define QDS_COLD inline
#endif

namespace qds {

constexpr int kRing1 = 5;   // K1 ring slots: columns L-2 .. L in use, L+1, L+2 in flight
constexpr int kRing2 = 4;   // K2 ring slots: columns L-1, L in use, L+1, L+2 in flight
constexpr int kHalo1 = 3;   // K1 radial halo rows on each side of a band
constexpr int kHalo2 = 2;   // K2 radial halo rows
constexpr int kPlanes = 9;  // planes per ring slot (K1: TRP..TAM; K2: TRP1..BX1, j_a x, r, theta)

// One CTA's work: instance, owned rows [r0, r1), first ring row rb0, owned
// columns [xa, xb).
struct MarchItem {
  int inst, r0, r1, rb0, xa, xb, pad0, pad1;
};

// Intermediate plane groups of K1 (K2 uses X_EXN only).  Each group holds
// `slots` copies of `planes` plane columns [mode][ring row].
enum {
  X_EXN = 0,  // 3 x {E_x, B_x at n+1/2} per face
  X_AF,       // 3 x {B_x at n (mean of the levels n -+ 1/2), E_r, E_theta (x-means of the old T)} per face
  X_CC,       // 2 x {T_r+, T_r-, T_th+, T_th- old + new; T_a+ + T_a- old + new; T_a+ new; T_a- new} per cell
  X_PH,       // 1 x {phi^n, phi^(n+1)} per face
  X_XS,       // axion source inputs of face L-1: E_x mean, T_r+, T_r- x-means, T_th+-, T_th- cell sums
  X_ST,       // S_a of face L-1
  N_X
};

struct MarchGeo {
  int RB;        // ring rows (threads per mode)
  int PL;        // elements per plane column (M * RB)
  int SS;        // elements per ring slot (rounded to 128 bytes)
  int NS;        // ring slots
  int off[N_X];  // element offsets of the intermediate groups
  int off_bar;   // byte offset of the mbarriers
  int bytes;     // dynamic shared memory
};

template <class R>
QDS_HD MarchGeo march_geo(int kind, int M, int RB) {
  MarchGeo g;
  g.RB = RB;
  g.PL = M * RB;
  const int per128 = 128 / (int)sizeof(C<R>);
  g.SS = (kPlanes * g.PL + per128 - 1) / per128 * per128;
  g.NS = kind == 0 ? kRing1 : kRing2;
  int o = g.NS * g.SS;
  for (int q = 0; q < N_X; q++) g.off[q] = o;
  g.off[X_EXN] = o; o += 3 * 2 * g.PL;
  if (kind == 0) {
    g.off[X_AF] = o; o += 3 * 3 * g.PL;
    g.off[X_CC] = o; o += 2 * 7 * g.PL;
    g.off[X_PH] = o; o += 2 * g.PL;
    g.off[X_XS] = o; o += 5 * g.PL;
    g.off[X_ST] = o; o += g.PL;
  }
  int b = o * (int)sizeof(C<R>);
  b = (b + 15) / 16 * 16;
  g.off_bar = b;
  g.bytes = b + g.NS * 8;
  return g;
}

// Bands of rows of one instance for a kernel with ring rows RB and radial
// halo `halo`: emit(r0, r1, rb0) per band.  One band when the grid fits;
// otherwise the first band starts at row 0 with no halo below, and every
// later band keeps `halo` rows below (its first ring row rounded down to
// even: the bulk copy's row coordinate times 8 bytes must be a multiple of
// 16) and `halo` rows above.  Needs RB >= 2 halo + 2.
template <class F>
inline void march_bands(int nr, int RB, int halo, F &&emit) {
  if (nr <= RB) {
    emit(0, nr, 0);
    return;
  }
  int r1 = RB - halo;
  emit(0, r1, 0);
  while (r1 < nr) {
    const int r0 = r1;
    const int rb0 = (r0 - halo) & ~1;
    r1 = rb0 + RB - halo < nr ? rb0 + RB - halo : nr;
    emit(r0, r1, rb0);
  }
}

// Shared-memory plan of a march CTA with RB ring rows, as compile-time
// constants (element offsets; the same numbers as march_geo).
template <class R, int M, int RB, int KIND>
struct MarchShape {
  static constexpr int PL = M * RB;
  static constexpr int per128 = 128 / (int)sizeof(C<R>);
  static constexpr int SS = (kPlanes * PL + per128 - 1) / per128 * per128;
  static constexpr int NS = KIND == 0 ? kRing1 : kRing2;
  static constexpr int O_EXN = NS * SS;
  static constexpr int O_AF = O_EXN + 6 * PL;
  static constexpr int O_CC = O_AF + (KIND == 0 ? 9 * PL : 0);
  static constexpr int O_PH = O_CC + (KIND == 0 ? 14 * PL : 0);
  static constexpr int O_XS = O_PH + (KIND == 0 ? 2 * PL : 0);
  static constexpr int O_ST = O_XS + (KIND == 0 ? 5 * PL : 0);
};

// Everything one thread of a march CTA needs: the instance, the CTA's band
// and segment, its shared memory, its own row and mode and their factors,
// and (set by iter) its elements of the ring slots and intermediate slots of
// the current iteration.  Element offsets within one instance fit in 32 bits
// (checked at create).
template <class R, int M, int RB_, int KIND>
struct MarchCtx : MarchShape<R, M, RB_, KIND> {
  using Sh = MarchShape<R, M, RB_, KIND>;
  static constexpr int RB = RB_;
  // instance
  int nx, nr, J, ld;
  bool per, closed, mw, ax;
  int s;                            // ring offset of the window
  size_t P;                         // elements per field (M planes)
  R h, dr, ih, idr, ma2, gs, gj;
  const C<R> *jx, *jr, *jt, *sext;  // this step's sources [M][nx][nr] in window order (may be null)
  const C<R> *in_rp, *in_tm;        // this step's injection at x_min, [M][nr] (may be null)
  const C<R> *o;                    // old state (global; phi_prev)
  C<R> *n;                          // new state (global)
  C<R> *scr;                        // scratch planes (global; j_a in planes 1..3)
  // CTA
  int rb0, r0, r1, xa, xb, L0;
  unsigned P32, ld32;               // elements per field, row stride
  C<R> *sm;                         // shared memory
  // thread
  int k, lr, j, off_t, koff;        // mode, ring row, row, k RB + lr, k RB
  unsigned gk;                      // global offset of the thread's mode and row in a field: k nx ld + j
  R irj, irh, kirj, kirh;           // 1/r_j, 1/r_{j+1/2}, k/r_j, k/r_{j+1/2}
  // iteration L (iter): the thread's elements of ring column L-d (rc[d]),
  // and of the intermediate slots of face / cell L-d: E_x, B_x at n+1/2
  // (ex[d]), the face quantities of the axion terms (af[d]), the cell values
  // of the axion current (cc[d]), phi (ph[d])
  const C<R> *rc[4];
  C<R> *ex[4], *af[4], *cc[4], *ph[4];
#if defined(QDS_EMU)
  size_t state_len;                 // bounds of the emulated global state
#endif

  QDS_HD void iter(int L) {
    const int q = L - L0;
#pragma unroll
    for (int d = 0; d < 4; d++) {
      rc[d] = sm + ((q - d + 4 * Sh::NS) % Sh::NS) * Sh::SS + off_t;
      const int t3 = (q - d + 12) % 3, t2 = (q - d + 12) % 2;
      ex[d] = sm + Sh::O_EXN + t3 * 2 * Sh::PL + off_t;
      af[d] = sm + Sh::O_AF + t3 * 3 * Sh::PL + off_t;
      // cell L-3 is read (phase 2) before cell L-1 is written (phase 3) in
      // the same slot; likewise phi of faces L-3 and L-2
      cc[d] = sm + Sh::O_CC + t2 * 7 * Sh::PL + off_t;
      ph[d] = sm + Sh::O_PH + off_t;
    }
  }
  QDS_HD bool cell_ok(int w) const { return per || (w >= 0 && w < nx); }
  QDS_HD bool face_ok(int w) const { return per || (w >= 0 && w <= nx - 2); }
  // storage slot of window column w (w inside the window, or any w when periodic)
  QDS_HD int slot(int w) const {
    if (per) { w %= nx; if (w < 0) w += nx; return w; }
    int q = w + s;
    return q >= nx ? q - nx : q;
  }
  QDS_HD C<R> srcv(const C<R> *a, int kk, int w, int jj) const {
    if (!a || !cell_ok(w) || jj < 0 || jj >= nr) return zero<R>();
    if (per) { w %= nx; if (w < 0) w += nx; }
    return ldg(a + ((size_t)kk * nx + w) * nr + jj);
  }
  // the caller's cell currents j_r, j_theta averaged onto face w (Eq. discrete_continuity positions)
  QDS_HD C<R> face_avg(const C<R> *a, int kk, int w, int jj) const {
    if (!a) return zero<R>();
    return R(0.5) * (srcv(a, kk, w, jj) + srcv(a, kk, w + 1, jj));
  }
  QDS_HD bool owned(int w, int jj) const { return w >= xa && w < xb && jj >= r0 && jj < r1; }
  // global offset of the thread's element of column w in a field plane set
  QDS_HD unsigned gcol(int w) const { return (unsigned)slot(w) * ld32 + gk; }
  // store the thread's element of window column w of a field of the new
  // state (gw = gcol(w)); the rear column becomes the (empty) front one when
  // the window moves
  QDS_HD void store(int field, int w, unsigned gw, C<R> v) const {
    if (mw && w == 0) v = zero<R>();
#if defined(QDS_EMU)
    QDS_CHECK((size_t)field * P32 + gw < state_len && j >= 0 && j < nr, "march store");
#endif
    n[(unsigned)field * P32 + gw] = v;
  }
  QDS_HD C<R> prev(int kk, int w) const {
    if (!face_ok(w)) return zero<R>();
    return ldg(o + (size_t)NFIELD * P + (size_t)kk * nx + slot(w));
  }
};

// ---------------------------------------------------------------------------
// Longitudinal leapfrog of one (row, mode) at face f from the ring columns of
// cells f (a) and f+1 (b): planes 0..3 T_r+, T_r-, T_th+, T_th-, 4 E_x, 5 B_x
// of the group.  The radial operators are in conservative form
// (1/r) d(r F)/dr = (r_+ F_+ - r_- F_-)/(r dr), algebraically the paper's
// average-plus-centred-difference form.  jxv: j_x at (f, j); jtf: j_theta
// at (f, J) (outer half row only).
// ---------------------------------------------------------------------------
template <class R>
struct Leap {
  C<R> ex, bx;        // E_x, B_x at n+1/2
  C<R> rp, rm, qp, qm;  // cell sums over f, f+1 of T_r+, T_r-, T_th+, T_th- (old)
  C<R> e0, b0;        // E_x, B_x at n-1/2
};

// B_x on the outer half row J: box scheme of Eq. em_r_open_bx over
// [r_{J-1/2}, r_{J+1/2}] x [t^{n-1/2}, t^{n+1/2}], right side at
// (x_{f+1/2}, r_J, t^n); the interior B_x one half row in, at n+1/2, enters
// the box.  a, b: the ring elements of cells f, f+1 on row J; er, eth: the
// x-means of E_r, E_theta on row J; b0: B_x at n-1/2.  (Arguments by value:
// the function is kept out of line.)
template <class R>
QDS_COLD C<R> leap_outer(const C<R> *a, const C<R> *b, int PL, int J, int k, R dr, R h, R ih, R idr, C<R> jtf,
                         C<R> er, C<R> eth, C<R> b0) {
  const C<R> rp1 = a[-1] + b[-1], rm1 = a[PL - 1] + b[PL - 1];
  const C<R> qp1 = a[2 * PL - 1] + b[2 * PL - 1], qm1 = a[3 * PL - 1] + b[3 * PL - 1];
  const C<R> er1 = R(0.25) * (rp1 + rm1), eth1 = R(0.25) * (qp1 + qm1);
  const R irh1 = R(1) / ((R(J) - R(0.5)) * dr);
  const C<R> bi = a[5 * PL - 1];
  const C<R> bin = bi - h * ((R(J) * eth - R(J - 1) * eth1) * irh1 + imul(R(k) * irh1, er1));
  const C<R> dxbr = (R(0.5) * ih) * ((b[2 * PL] - b[3 * PL]) - (a[2 * PL] - a[3 * PL]));
  const C<R> ero = R(0.5) * (er1 + er);
  const R rJ = R(J) * dr;
  const C<R> rhs = R(0.5) * dxbr - (R(0.5) / rJ) * (eth + imul(R(k), ero)) - R(0.5) * jtf;
  const R A_ = R(0.5) * ih, B_ = R(0.5) * idr;
  return (rhs - (A_ - B_) * bin + (A_ - B_) * b0 + (A_ + B_) * bi) * (R(1) / (A_ + B_));
}

// OUTER: the thread on the outer half row also forms B_x there (K2); in K1
// that value is left to the CTA's boundary warp (outer_p1) and the thread
// returns B_x unset.
template <class R, int M, int RB, int KIND, bool OUTER = true>
QDS_HD void em_leap(const MarchCtx<R, M, RB, KIND> &c, const C<R> *a, const C<R> *b, C<R> jxv, C<R> jtf, Leap<R> &o) {
  const int j = c.j, k = c.k; constexpr int PL = M * RB;
  o.rp = a[0] + b[0];
  o.rm = a[PL] + b[PL];
  o.qp = a[2 * PL] + b[2 * PL];
  o.qm = a[3 * PL] + b[3 * PL];
  o.e0 = a[4 * PL];
  o.b0 = a[5 * PL];
  const C<R> er = R(0.25) * (o.rp + o.rm), bth = R(0.25) * (o.rp - o.rm);
  const C<R> eth = R(0.25) * (o.qp + o.qm), brr = R(0.25) * (o.qp - o.qm);
  // E_x: (1/r) d(r B_theta)/dr + i (m/r) B_r - j_x (Eq. Gammax_explicit);
  // on the axis only m = 0, from B_theta of the first half row (Eq. axis_Ex)
  if (j == 0) {
    o.ex = (k != 0) ? zero<R>() : o.e0 + c.h * (R(4) * c.idr * bth - jxv);
  } else {
    const C<R> blo = R(0.25) * ((a[-1] + b[-1]) - (a[PL - 1] + b[PL - 1]));
    const C<R> curl = ((R(j) + R(0.5)) * bth - (R(j) - R(0.5)) * blo) * c.irj;
    o.ex = o.e0 + c.h * (curl + imul(c.kirj, brr) - jxv);
  }
  if (j == c.J && !c.closed) {
    if (OUTER) o.bx = leap_outer<R>(a, b, PL, c.J, k, c.dr, c.h, c.ih, c.idr, jtf, er, eth, o.b0);
    else o.bx = zero<R>();
  } else {
    // B_x: -(1/r) d(r E_theta)/dr - i (m/r) E_r (Eq. Phix_explicit)
    C<R> ehi = zero<R>();
    if (j + 1 < c.nr) ehi = R(0.25) * (a[2 * PL + 1] + b[2 * PL + 1] + a[3 * PL + 1] + b[3 * PL + 1]);
    const C<R> curl = (R(j + 1) * ehi - R(j) * eth) * c.irh;
    o.bx = o.b0 - c.h * (curl + imul(c.kirh, er));
  }
}

// ---------------------------------------------------------------------------
// Characteristic shift of one (row, mode) at cell cc (Eqs. Trp_update,
// Trm_update, Ttp_update, Ttm_update, axis_Ttheta; the outer half row by the
// box scheme of Eq. em_r_open_bt).  A, B, Cc: the thread's ring elements of
// cells cc-1, cc, cc+1; ea, eb: its elements of the new E_x, B_x at faces
// cc-1 and cc.  CUR supplies the face currents:
//   jr(face, row), jt(face, row), jx(face, row).
// ---------------------------------------------------------------------------
template <class R>
struct Shift {
  C<R> tp, tm, up, um;
};

// T_r+- on the outer half row J: E_r by the shift with the Gamma_r source
// alone, B_theta by the box scheme of Eq. em_r_open_bt over [r_{J-1/2},
// r_{J+1/2}] x [t^n, t^{n+1}] with its right side from time-n fields; the
// interior B_theta one half row in, at n+1, enters the box.  a*, b*, n*: the
// old T_r+- (p, m) and T_th+- (tp, tm) of cells cc-1, cc, cc+1 on row J (1:
// row J-1); ea, eb: E_x, B_x at n+1/2 of faces cc-1, cc on row J; jr_* /
// jx_*: the face currents (l: face cc-1, r: face cc; 1: row J-1), zero at a
// face that is not live.  (Arguments by value: the function is kept out of
// line.)
template <class R>
struct Pair {
  C<R> a, b;
};
template <class R>
QDS_COLD Pair<R> shift_outer(C<R> ap1, C<R> am1, C<R> ap, C<R> am, C<R> bp1, C<R> bm1, C<R> bp, C<R> bm, C<R> btp,
                             C<R> btm, C<R> np1, C<R> nm1, C<R> np, C<R> nm, const C<R> *ea, const C<R> *eb, int PL,
                             int J, int k, R dr, R h, R ih, R idr, R kirh, bool fa, bool fb, C<R> jr_l1, C<R> jr_l,
                             C<R> jr_r1, C<R> jr_r, C<R> jx_l, C<R> jx_r) {
  const R irh1 = R(1) / ((R(J) - R(0.5)) * dr), kirh1 = R(k) * irh1;
  C<R> sp1 = zero<R>(), sm1 = zero<R>(), gl = zero<R>(), gr = zero<R>();
  if (fa) {
    sp1 = -imul(kirh1, ea[PL - 1]) - jr_l1 + idr * (ea[0] - ea[-1]);
    gl = -imul(kirh, ea[PL]) - jr_l;
  }
  if (fb) {
    sm1 = -imul(kirh1, eb[PL - 1]) - jr_r1 - idr * (eb[0] - eb[-1]);
    gr = -imul(kirh, eb[PL]) - jr_r;
  }
  const C<R> ip = ap1 + h * sp1, im = nm1 + h * sm1;
  const C<R> btin = R(0.5) * (ip - im);
  const C<R> ernew = R(0.5) * (ap + nm + h * (gl + gr));
  const C<R> erl = R(0.25) * ((ap1 + am1) + (ap + am));
  const C<R> err = R(0.25) * ((np1 + nm1) + (np + nm));
  const C<R> bo = R(0.5) * (bp - bm), bi = R(0.5) * (bp1 - bm1);
  const C<R> bth = R(0.5) * (bi + bo);
  const C<R> br = R(0.5) * (btp - btm);
  const R rJ = R(J) * dr;
  const C<R> rhs = (R(-0.25) * ih) * (err - erl) - (R(0.5) / rJ) * (bth + imul(R(k), br)) + R(0.25) * (jx_l + jx_r);
  const R A_ = R(0.5) * ih, B_ = R(0.5) * idr;
  const C<R> btn = (rhs - (A_ - B_) * btin + (A_ - B_) * bo + (A_ + B_) * bi) * (R(1) / (A_ + B_));
  Pair<R> o;
  o.a = ernew + btn;
  o.b = ernew - btn;
  return o;
}

// Old T of the cells cc-1 (a), cc (b), cc+1 (n) that the shift reads:
// plane 0..3 = T_r+, T_r-, T_th+, T_th-; dj = 0 (the thread's row) or -1 (the
// row below, outer half row only).  From the ring columns:
template <class R, int PL>
struct CellsRing {
  const C<R> *A, *B, *Cc;
  QDS_HD C<R> a(int p, int dj) const { return A[p * PL + dj]; }
  QDS_HD C<R> b(int p, int dj) const { return B[p * PL + dj]; }
  QDS_HD C<R> n(int p, int dj) const { return Cc[p * PL + dj]; }
};

// OUTER: as for em_leap (T_r+- of the outer half row in K1 come from the
// boundary warp, outer_p3; the thread returns them unset).
template <class R, int M, int RB, int KIND, class CELLS, class CUR, bool OUTER = true>
QDS_HD void em_shift(const MarchCtx<R, M, RB, KIND> &c, int cc, const CELLS &cl, const C<R> *ea, const C<R> *eb,
                     const CUR &cur, Shift<R> &o) {
  const int j = c.j, k = c.k; constexpr int PL = M * RB;
  const bool fa = c.face_ok(cc - 1), fb = c.face_ok(cc);
  if (j < c.J || c.closed) {
    // T_r+ from cell cc-1 through face cc-1, T_r- from cell cc+1 through
    // face cc: Gamma_r = -i (m/r) B_x - j_r, Phi_r = dE_x/dr
    C<R> sp = zero<R>(), sm = zero<R>();
    if (fa) {
      const C<R> ehi = (j + 1 < c.nr) ? ea[1] : zero<R>();
      sp = -imul(c.kirh, ea[PL]) - cur.jr(cc - 1, j) + c.idr * (ehi - ea[0]);
    }
    if (fb) {
      const C<R> ehi = (j + 1 < c.nr) ? eb[1] : zero<R>();
      sm = -imul(c.kirh, eb[PL]) - cur.jr(cc, j) - c.idr * (ehi - eb[0]);
    }
    o.tp = cl.a(0, 0) + c.h * sp;
    o.tm = cl.n(1, 0) + c.h * sm;
  } else if (!OUTER) {
    o.tp = o.tm = zero<R>();
  } else {
    const int J = c.J;
    const C<R> z = zero<R>();
    const Pair<R> t = shift_outer<R>(
        cl.a(0, -1), cl.a(1, -1), cl.a(0, 0), cl.a(1, 0), cl.b(0, -1), cl.b(1, -1), cl.b(0, 0), cl.b(1, 0),
        cl.b(2, 0), cl.b(3, 0), cl.n(0, -1), cl.n(1, -1), cl.n(0, 0), cl.n(1, 0), ea, eb, PL, J, k, c.dr, c.h,
        c.ih, c.idr, c.kirh, fa, fb, fa ? cur.jr(cc - 1, J - 1) : z, fa ? cur.jr(cc - 1, J) : z,
        fb ? cur.jr(cc, J - 1) : z, fb ? cur.jr(cc, J) : z, fa ? cur.jx(cc - 1, J) : z, fb ? cur.jx(cc, J) : z);
    o.tp = t.a;
    o.tm = t.b;
  }
  // T_th+ from cell cc+1 through face cc, T_th- from cell cc-1 through face
  // cc-1: Gamma_th = -dB_x/dr - j_theta, Phi_th = i (m/r) E_x; on the axis
  // only m = 1 (Eq. axis_Ttheta)
  if (j == 0 && k != 1) {
    o.up = zero<R>();
    o.um = zero<R>();
    return;
  }
  C<R> sp = zero<R>(), sm = zero<R>();
  if (fb) {
    C<R> g, p;
    if (j == 0) {
      g = -(R(2) * c.idr) * eb[PL] - cur.jt(cc, 0);
      p = imul(c.idr, eb[1] - eb[0]);
    } else {
      g = -c.idr * (eb[PL] - eb[PL - 1]) - cur.jt(cc, j);
      p = imul(c.kirj, eb[0]);
    }
    sp = g + p;
  }
  if (fa) {
    C<R> g, p;
    if (j == 0) {
      g = -(R(2) * c.idr) * ea[PL] - cur.jt(cc - 1, 0);
      p = imul(c.idr, ea[1] - ea[0]);
    } else {
      g = -c.idr * (ea[PL] - ea[PL - 1]) - cur.jt(cc - 1, j);
      p = imul(c.kirj, ea[0]);
    }
    sm = g - p;
  }
  o.up = cl.n(2, 0) + c.h * sp;
  o.um = cl.a(3, 0) + c.h * sm;
}

// Face currents of the EM field: the caller's arrays (j_x at faces, j_r and
// j_theta at cells, x-averaged onto the faces).
template <class R, int M, int RB>
struct CurCaller {
  const MarchCtx<R, M, RB, 0> &c;
  QDS_HD C<R> jx(int w, int jj) const { return c.srcv(c.jx, c.k, w, jj); }
  QDS_HD C<R> jr(int w, int jj) const { return c.face_avg(c.jr, c.k, w, jj); }
  QDS_HD C<R> jt(int w, int jj) const { return c.face_avg(c.jt, c.k, w, jj); }
};

// Face currents of the regenerated field: j_a at faces, from the K2 ring
// (planes 6, 7, 8 of the column of the face); fa / fb are the thread's ring
// elements of the columns of faces cc-1 and cc.
template <class R, int M, int RB>
struct CurAxion {
  const MarchCtx<R, M, RB, 1> &c;
  const C<R> *fa, *fb;
  int cc;
  QDS_HD const C<R> *at(int w, int jj) const { return (w == cc ? fb : fa) + (jj - c.j); }
  QDS_HD C<R> jx(int w, int jj) const { return at(w, jj)[6 * M * RB]; }
  QDS_HD C<R> jr(int w, int jj) const { return at(w, jj)[7 * M * RB]; }
  QDS_HD C<R> jt(int w, int jj) const { return at(w, jj)[8 * M * RB]; }
};

// ---------------------------------------------------------------------------
// Sum over three pairs of the mode convolution (Eq. mode_convolution) for
// output mode m, modes 0..M-1 retained, negative modes the conjugates (Eq.
// fourier_decomp):
//   m = 0:  A_0 B_0 + (1/2) sum_{k>=1} Re(A_k conj B_k)
//   m > 0:  (1/2) [ sum_{k+l=m} A_k B_l + sum_{k-l=m} A_k conj B_l
//                   + sum_{l-k=m} conj A_k B_l ]
// written as fused multiply-adds on the real and imaginary parts.
// ---------------------------------------------------------------------------
template <class R>
QDS_HD R fmr(R a, R b, R c) {
#if defined(__CUDA_ARCH__)
  return fma(a, b, c);
#else
  return std::fma(a, b, c);
#endif
}
template <class R>
QDS_HD void cmac(R &sr, R &si, C<R> a, C<R> b) {  // += a b
  sr = fmr(a.re, b.re, sr); sr = fmr(-a.im, b.im, sr);
  si = fmr(a.re, b.im, si); si = fmr(a.im, b.re, si);
}
template <class R>
QDS_HD void cmac_cb(R &sr, R &si, C<R> a, C<R> b) {  // += a conj(b)
  sr = fmr(a.re, b.re, sr); sr = fmr(a.im, b.im, sr);
  si = fmr(a.im, b.re, si); si = fmr(-a.re, b.im, si);
}
template <class R>
QDS_HD void cmac_ca(R &sr, R &si, C<R> a, C<R> b) {  // += conj(a) b
  sr = fmr(a.re, b.re, sr); sr = fmr(a.im, b.im, sr);
  si = fmr(a.re, b.im, si); si = fmr(-a.im, b.re, si);
}

template <class R, int M>
QDS_HD C<R> conv3(int m, const C<R> (&A)[3][M], const C<R> (&B)[3][M]) {
  // one accumulator pair per convolution pair: independent FMA chains
  R sr[3], si[3];
#pragma unroll
  for (int p = 0; p < 3; p++) { sr[p] = R(0); si[p] = R(0); }
  if (m == 0) {
    R hr[3];
#pragma unroll
    for (int p = 0; p < 3; p++) {
      hr[p] = R(0);
      cmac(sr[p], si[p], A[p][0], B[p][0]);
#pragma unroll
      for (int k = 1; k < M; k++) { hr[p] = fmr(A[p][k].re, B[p][k].re, hr[p]); hr[p] = fmr(A[p][k].im, B[p][k].im, hr[p]); }
    }
    return mk<R>(fmr(R(0.5), (hr[0] + hr[1]) + hr[2], (sr[0] + sr[1]) + sr[2]), (si[0] + si[1]) + si[2]);
  }
#pragma unroll
  for (int p = 0; p < 3; p++) {
#pragma unroll
    for (int k = 0; k < M; k++) {
      if (k <= m && m - k < M) cmac(sr[p], si[p], A[p][k], B[p][m - k]);  // k + l = m
      if (k - m >= 0) cmac_cb(sr[p], si[p], A[p][k], B[p][k - m]);       // k - l = m
      if (k + m < M) cmac_ca(sr[p], si[p], A[p][k], B[p][k + m]);        // l - k = m
    }
  }
  return mk<R>(R(0.5) * ((sr[0] + sr[1]) + sr[2]), R(0.5) * ((si[0] + si[1]) + si[2]));
}

// ---------------------------------------------------------------------------
// Laser injection at x_min: the ring slot of window column -1 (read as zeros
// by the bulk copy: the open boundary of Eq. em_x_open) takes the injected
// inflow T_r^+ and T_th^- of the EM field on the thread's row, before the
// shift into cell 0 reads it (two iterations later).
// ---------------------------------------------------------------------------
template <class R, int M, int RB>
QDS_HD void k1_inflow(const MarchCtx<R, M, RB, 0> &c, int L) {
  if (L != -1 || c.per || c.j >= c.nr || (!c.in_rp && !c.in_tm)) return;
  C<R> *p = const_cast<C<R> *>(c.rc[0]);
  const size_t q = (size_t)c.k * c.nr + c.j;
  p[0] = c.in_rp ? ldg(c.in_rp + q) : zero<R>();
  p[3 * M * RB] = c.in_tm ? ldg(c.in_tm + q) : zero<R>();
}

// ---------------------------------------------------------------------------
// K1 phase 1: A at face L-1 on rows [r0-2, r1+2).
// ---------------------------------------------------------------------------
template <class R, int M, int RB>
QDS_HD void k1_p1(const MarchCtx<R, M, RB, 0> &c, int L) {
  const int j = c.j, k = c.k; constexpr int PL = M * RB;
  if (L < c.xa || L > c.xb + 1) return;
  if (j < c.r0 - 2 || j >= c.r1 + 2 || j < 0 || j >= c.nr) return;
  const int f = L - 1;
  C<R> *ex = c.ex[1];
  const bool own = c.owned(f, j);
  const unsigned gw = own ? c.gcol(f) : 0u;
  if (!c.face_ok(f)) {
    // the held-zero face nx-1 (its consumers test face_ok themselves)
    ex[0] = zero<R>();
    ex[PL] = zero<R>();
    if (own) {
      c.store(EX, f, gw, zero<R>());
      c.store(BX, f, gw, zero<R>());
    }
    return;
  }
  const C<R> jxv = c.srcv(c.jx, k, f, j);
  const C<R> jtf = (j == c.J && !c.closed) ? c.face_avg(c.jt, k, f, j) : zero<R>();
  Leap<R> o;
  em_leap<R, M, RB, 0, false>(c, c.rc[1], c.rc[0], jxv, jtf, o);
  const bool outer = j == c.J && !c.closed;  // B_x there: the boundary warp (outer_p1)
  ex[0] = o.ex;
  if (!outer) ex[PL] = o.bx;
  if (c.ax) {
    C<R> *af = c.af[1];
    C<R> *xs = c.sm + c.O_XS + c.off_t;
    if (!outer) af[0] = R(0.5) * (o.b0 + o.bx);  // B_x at n
    af[PL] = R(0.25) * (o.rp + o.rm);      // E_r, x-mean over cells f, f+1
    af[2 * PL] = R(0.25) * (o.qp + o.qm);  // E_theta
    xs[0] = R(0.5) * (o.e0 + o.ex);        // E_x at n
    xs[PL] = R(0.5) * o.rp;
    xs[2 * PL] = R(0.5) * o.rm;
    xs[3 * PL] = o.qp;
    xs[4 * PL] = o.qm;
  }
  if (own) {
    c.store(EX, f, gw, o.ex);
    if (!outer) c.store(BX, f, gw, o.bx);
  }
}

// ---------------------------------------------------------------------------
// K1 phase 2, task S: the inputs of S_a at face f = L-1 for the thread's row
// (rows [r0-1, r1+1)), as three convolution pairs.  Every field is averaged
// onto (x_{f+1/2}, r_{j+1/2}); E_x, B_x also over the levels n -+ 1/2.  The
// transverse term is written in transport variables: with E_r, B_theta from
// the same x-average of T_r and E_theta, B_r from the same four-point average
// of T_theta, the symmetry of C_m gives
//   C{E_r,B_r} + C{E_th,B_th} = (1/2)(C{T_r+,T_th+} - C{T_r-,T_th-}),
// free of the cancellation of E.B between co-propagating waves (Eq.
// mixing_source: zero in vacuum).  Beyond the last half row the averages use
// zero-gradient extrapolation (open) or zero (closed).
//   S_a = C{E_x, B_x} + (1/2) C{T_r+, T_th+} - (1/2) C{T_r-, T_th-}
// (the weights 1/2 are folded into the first factors).
// ---------------------------------------------------------------------------
template <class R, int M, int RB>
QDS_HD void k1_inputs_s(const MarchCtx<R, M, RB, 0> &c, int f, C<R> (&A)[3][M], C<R> (&B)[3][M]) {
  const int j = c.j; constexpr int PL = M * RB;
  const C<R> *xs = c.sm + c.O_XS + c.lr;
  const C<R> *af = c.af[1] - c.koff;  // face f = L-1
  const bool top = j == c.J;
  const R wt = top ? (c.closed ? R(0.5) : R(1)) : R(0.5);  // E_x mean weight of row j when row j+1 is missing
  const R wq = top ? (c.closed ? R(0.25) : R(0.5)) : R(0.25);
#pragma unroll
  for (int kk = 0; kk < M; kk++) {
    const int o = kk * RB;
    if (!top) {
      A[0][kk] = R(0.5) * (xs[o] + xs[o + 1]);
      B[1][kk] = R(0.25) * (xs[3 * PL + o] + xs[3 * PL + o + 1]);
      B[2][kk] = R(0.25) * (xs[4 * PL + o] + xs[4 * PL + o + 1]);
    } else {
      A[0][kk] = wt * xs[o];
      B[1][kk] = wq * xs[3 * PL + o];
      B[2][kk] = wq * xs[4 * PL + o];
    }
    B[0][kk] = af[o];
    A[1][kk] = R(0.5) * xs[PL + o];
    A[2][kk] = R(-0.5) * xs[2 * PL + o];
  }
}

// ---------------------------------------------------------------------------
// K1 phase 2, tasks Dx, Dr, Dth: the inputs of one component of the axion
// current j_a = g (B0 d_t phi - E0 x grad phi) (Eqs. jax_mode, jar_mode,
// jat_mode) at face f = L-3 for the thread's row, as three convolution pairs
// (weights folded into the first factors), with (d_theta phi)^(l) = -i l phi^(l):
//   j_a,x at (x_{f+1/2}, r_j, t^n), j_a,r at (x_{f+1/2}, r_{j+1/2}, t^{n+1/2}),
//   j_a,theta at (x_{f+1/2}, r_j, t^{n+1/2});
// d_t phi = (c/2)(T_a+ + T_a-), d_x phi = (1/2)(T_a- - T_a+) (Eq. phi_update).
// Below the axis a half-row scalar mirrors with parity (-1)^l; E_r and
// B_theta below the axis follow the T_r ghost of Eq. axis_Tr.  In terms of
// transport variables at n+1/2 (means of the levels n and n+1):
//   C{B_r, d_t phi} - C{E_th, d_x phi} = (1/2)(C{T_th+, T_a+} - C{T_th-, T_a-}),
//   C{B_th, d_t phi} + C{E_r, d_x phi} = (1/2)(C{T_r+, T_a-} - C{T_r-, T_a+}).
// ---------------------------------------------------------------------------
template <class R, int M, int RB>
QDS_HD void k1_inputs_d(const MarchCtx<R, M, RB, 0> &c, int f, int comp, C<R> (&A)[3][M], C<R> (&B)[3][M]) {
  const int j = c.j; constexpr int PL = M * RB;
  // face f = L-3 and cells f, f+1 = L-3, L-2
  const C<R> *af = c.af[3] - c.koff;
  const C<R> *cf = c.cc[3] - c.koff;
  const C<R> *cg = c.cc[2] - c.koff;
  const C<R> *ph = c.ph[3] - c.koff;
  const C<R> *ex = c.ex[3] - c.koff;
  const bool top = j == c.J;
  if (comp == 0) {
    // j_a,x = g (C{B_x, d_t phi} - C{E_r, (d_theta phi)/r} + C{E_theta, d_r phi})
#pragma unroll
    for (int kk = 0; kk < M; kk++) {
      const int o = kk * RB;
      const R par = (kk & 1) ? R(-1) : R(1);
      const C<R> bxh = af[o];
      const C<R> bxl = (j > 0) ? af[o - 1] : par * bxh;
      A[0][kk] = R(0.5) * (bxl + bxh);
      const C<R> dth = R(0.125) * (cf[4 * PL + o] + cg[4 * PL + o]);
      const C<R> dtl = (j > 0) ? R(0.125) * (cf[4 * PL + o - 1] + cg[4 * PL + o - 1]) : par * dth;
      B[0][kk] = R(0.5) * (dtl + dth);
      const C<R> erh = af[PL + o];
      C<R> erl;
      if (j > 0) erl = af[PL + o - 1];
      else if (kk == 1) erl = imul(R(2), af[2 * PL + o]) - erh;
      else erl = -erh;
      A[1][kk] = R(-0.5) * (erl + erh);
      const C<R> p = ph[o];
      const C<R> pl = (j > 0) ? ph[o - 1] : par * p;
      if (j > 0) B[1][kk] = imul(-R(kk) * R(0.5) * c.irj, pl + p);
      else B[1][kk] = (kk == 1) ? imul(-c.idr, p - pl) : zero<R>();
      A[2][kk] = af[2 * PL + o];
      B[2][kk] = c.idr * (p - pl);
    }
  } else if (comp == 1) {
    // j_a,r = g ((1/2) C{T_th+, T_a+} - (1/2) C{T_th-, T_a-} + C{E_x, (d_theta phi)/r})
#pragma unroll
    for (int kk = 0; kk < M; kk++) {
      const int o = kk * RB;
      const C<R> p = R(0.5) * (cf[2 * PL + o] + cg[2 * PL + o]);
      const C<R> m_ = R(0.5) * (cf[3 * PL + o] + cg[3 * PL + o]);
      C<R> p1, m1;
      if (!top) {
        p1 = R(0.5) * (cf[2 * PL + o + 1] + cg[2 * PL + o + 1]);
        m1 = R(0.5) * (cf[3 * PL + o + 1] + cg[3 * PL + o + 1]);
      } else if (c.closed) {
        p1 = zero<R>();
        m1 = zero<R>();
      } else {
        p1 = p;
        m1 = m_;
      }
      A[0][kk] = R(0.125) * (p + p1);
      A[1][kk] = R(-0.125) * (m_ + m1);
      B[0][kk] = R(0.5) * (cf[5 * PL + o] + cg[5 * PL + o]);
      B[1][kk] = R(0.5) * (cf[6 * PL + o] + cg[6 * PL + o]);
      const C<R> exl = ex[o];
      const C<R> exh = !top ? ex[o + 1] : (c.closed ? zero<R>() : exl);
      A[2][kk] = R(0.5) * (exl + exh);
      B[2][kk] = imul(-R(kk) * R(0.5) * c.irh, ph[o] + ph[PL + o]);
    }
  } else {
    // j_a,theta = g ((1/2) C{T_r+, T_a-} - (1/2) C{T_r-, T_a+} - C{E_x, d_r phi})
#pragma unroll
    for (int kk = 0; kk < M; kk++) {
      const int o = kk * RB;
      const R par = (kk & 1) ? R(-1) : R(1);
      if (j > 0) {
        A[0][kk] = R(0.0625) * ((cf[o] + cg[o]) + (cf[o - 1] + cg[o - 1]));
        A[1][kk] = R(-0.0625) * ((cf[PL + o] + cg[PL + o]) + (cf[PL + o - 1] + cg[PL + o - 1]));
      } else if (kk == 1) {
        A[0][kk] = imul(R(0.125), cf[3 * PL + o] + cg[3 * PL + o]);
        A[1][kk] = imul(R(-0.125), cf[2 * PL + o] + cg[2 * PL + o]);
      } else {
        A[0][kk] = zero<R>();
        A[1][kk] = zero<R>();
      }
      const C<R> aph = R(0.5) * (cf[5 * PL + o] + cg[5 * PL + o]);
      const C<R> amh = R(0.5) * (cf[6 * PL + o] + cg[6 * PL + o]);
      const C<R> apl = (j > 0) ? R(0.5) * (cf[5 * PL + o - 1] + cg[5 * PL + o - 1]) : par * aph;
      const C<R> aml = (j > 0) ? R(0.5) * (cf[6 * PL + o - 1] + cg[6 * PL + o - 1]) : par * amh;
      B[0][kk] = R(0.5) * (aml + amh);
      B[1][kk] = R(0.5) * (apl + aph);
      A[2][kk] = -ex[o];
      const C<R> pbh = R(0.5) * (ph[o] + ph[PL + o]);
      const C<R> pbl = (j > 0) ? R(0.5) * (ph[o - 1] + ph[PL + o - 1]) : par * pbh;
      B[2][kk] = c.idr * (pbh - pbl);
    }
  }
}

// K1 phase 2: the convolution tasks of the thread's row (task t on the mode
// thread t mod M): t = 0 S_a of face L-1 into shared memory, t = 1..3 the
// components x, r, theta of j_a of face L-3 into the scratch planes.  All
// tasks share one convolution code path.
template <class R, int M, int RB>
QDS_HD void k1_p2(const MarchCtx<R, M, RB, 0> &c, int L, bool ar) {
  const int j = c.j;
#pragma unroll 1
  for (int t = c.k; t < 4; t += M) {
    int f;
    if (t == 0) {
      if (!c.ax || L < c.xa || L > c.xb + 1) continue;
      if (j < c.r0 - 1 || j >= c.r1 + 1 || j < 0 || j >= c.nr) continue;
      f = L - 1;
      if (!c.face_ok(f)) continue;  // Gamma_a there is zero without reading S_a
    } else {
      if (!ar || L < c.xa + 3 || L > c.xb + 2) continue;
      if (j < c.r0 || j >= c.r1 || j < 0 || j >= c.nr) continue;
      f = L - 3;
    }
    C<R> out[M];
    if (t > 0 && !c.face_ok(f)) {
#pragma unroll
      for (int m = 0; m < M; m++) out[m] = zero<R>();
    } else {
      C<R> A[3][M], B[3][M];
      if (t == 0) k1_inputs_s<R, M, RB>(c, f, A, B);
      else k1_inputs_d<R, M, RB>(c, f, t - 1, A, B);
#pragma unroll
      for (int m = 0; m < M; m++) out[m] = conv3<R, M>(m, A, B);
    }
    if (t == 0) {
      C<R> *st = c.sm + c.O_ST + c.lr;
#pragma unroll
      for (int m = 0; m < M; m++) {
        C<R> S = out[m];
        if (c.sext) S += c.srcv(c.sext, m, f, j);
        st[m * RB] = S;
      }
    } else {
      // j_a into scratch plane t (planes 1..3), every mode of the row
      const unsigned g0 = (unsigned)c.slot(f) * c.ld32 + (unsigned)j;
      const unsigned ms = (unsigned)c.nx * c.ld32;
#if defined(QDS_EMU)
      QDS_CHECK((size_t)t * c.P32 + g0 + (M - 1) * (size_t)ms < 4 * (size_t)c.P32, "j_a store");
#endif
      C<R> *out_g = c.scr + (unsigned)t * c.P32 + g0;
#pragma unroll
      for (int m = 0; m < M; m++) out_g[m * ms] = c.gj * out[m];
    }
  }
}

// Per-thread registers carried from one K1 iteration to the next.
template <class R>
struct K1Regs {
  C<R> gam_prev, gam;   // Gamma_a at faces L-2, L-1 (own row and mode)
  C<R> tap_prev, tam_prev;  // T_a+-^(n+1/2) at cell L-2
  bool bad;             // a stored value is not finite
};

// ---------------------------------------------------------------------------
// K1 phase 3: Gamma_a at face L-1 (rows [r0-1, r1+1)), the shift at cell
// L-1 (same rows), phi at face L-2 (rows [r0-1, r1)).
//   Gamma_a = (1/r) d/dr (r dphi/dr) - m^2 phi / r^2 - m_a^2 phi + g S_a;
// beyond the outermost half row the exterior phi comes from the outgoing
// condition (d_t + c d_r) phi = 0 centred at r_J (Eq. axion_r_ghost) with
// d_t phi taken half a step back.
// ---------------------------------------------------------------------------
template <class R, int M, int RB>
QDS_HD void k1_p3(const MarchCtx<R, M, RB, 0> &c, int L, K1Regs<R> &rg) {
  const int j = c.j, k = c.k; constexpr int PL = M * RB;
  const bool rows = j >= c.r0 - 1 && j < c.r1 + 1 && j >= 0 && j < c.nr;
  if (!rows) return;
  // Gamma_a at face L-1
  const int f = L - 1;
  rg.gam = zero<R>();
  if (c.ax && L >= c.xa && L <= c.xb + 1 && c.face_ok(f)) {
    const C<R> *a = c.rc[1] + 6 * PL;
    const C<R> pc = a[0];
    const C<R> pm = (j > 0) ? a[-1] : zero<R>();  // weight j = 0 on the axis
    C<R> pp;
    if (j < c.J) pp = a[1];
    else if (c.closed) pp = pc;
    else pp = a[-1] - (R(2) * c.dr * c.ih) * (pc - c.prev(k, f));
    const C<R> lap = (R(j + 1) * (pp - pc) - R(j) * (pc - pm)) * (c.idr * c.idr / (R(j) + R(0.5)));
    const C<R> S = c.sm[c.O_ST + c.off_t];
    rg.gam = lap - (c.kirh * c.kirh + c.ma2) * pc + c.gs * S;
  }
  // shift at cell cc = L-1
  C<R> ap = zero<R>(), am = zero<R>();
  if (L >= c.xa + 1 && L <= c.xb + 1) {
    const int cc = L - 1;
    const C<R> *A = c.rc[2], *B = c.rc[1], *Cn = c.rc[0];
    Shift<R> sh;
    sh.tp = sh.tm = sh.up = sh.um = zero<R>();
    if (c.cell_ok(cc)) {
      CurCaller<R, M, RB> cur{c};
      em_shift<R, M, RB, 0, CellsRing<R, M * RB>, CurCaller<R, M, RB>, false>(
          c, cc, CellsRing<R, M * RB>{A, B, Cn}, c.ex[2], c.ex[1], cur, sh);
      if (c.ax) {
        ap = A[7 * PL] + c.h * rg.gam_prev;
        am = Cn[8 * PL] + c.h * rg.gam;
      }
    }
    const bool outer = j == c.J && !c.closed;  // T_r+- there: the boundary warp (outer_p3)
    if (c.ax) {
      C<R> *cs = c.cc[1];
      if (!outer) {
        cs[0] = B[0] + sh.tp;
        cs[PL] = B[PL] + sh.tm;
      }
      cs[2 * PL] = B[2 * PL] + sh.up;
      cs[3 * PL] = B[3 * PL] + sh.um;
      cs[4 * PL] = (B[7 * PL] + B[8 * PL]) + (ap + am);
      cs[5 * PL] = ap;
      cs[6 * PL] = am;
    }
    if (c.owned(cc, j)) {
      const unsigned gw = c.gcol(cc);
      if (!outer) {
        c.store(TRP, cc, gw, sh.tp);
        c.store(TRM, cc, gw, sh.tm);
      }
      c.store(TTP, cc, gw, sh.up);
      c.store(TTM, cc, gw, sh.um);
      if (c.ax) {
        c.store(TAP, cc, gw, ap);
        c.store(TAM, cc, gw, am);
      }
      rg.bad = rg.bad || (!outer && !finite_c(sh.tp)) || !finite_c(ap);
    }
  }
  // phi at face L-2 from T_a^(n+1/2) of cells L-2 and L-1
  if (c.ax && L >= c.xa + 2 && L <= c.xb + 1 && j < c.r1) {
    const int fp = L - 2;
    C<R> po = zero<R>(), v = zero<R>();
    if (c.face_ok(fp)) {
      po = c.rc[2][6 * PL];
      v = po + (R(0.25) * c.h) * ((rg.tap_prev + rg.tam_prev) + (ap + am));
    }
    C<R> *p = c.ph[2];
    p[0] = po;
    p[PL] = v;
    if (c.owned(fp, j)) {
      c.store(PHI, fp, c.gcol(fp), v);
      if (j == c.J) {
        C<R> pv = po;
        if (c.mw && fp == 0) pv = zero<R>();
        const size_t q = (size_t)NFIELD * c.P32 + (size_t)k * c.nx + c.slot(fp);
#if defined(QDS_EMU)
        QDS_CHECK(q < c.state_len, "phi_prev store");
#endif
        c.n[q] = pv;
      }
    }
  }
  rg.gam_prev = rg.gam;
  rg.tap_prev = ap;
  rg.tam_prev = am;
}

// ---------------------------------------------------------------------------
// K1 boundary warp: lane k computes, for mode k, the values of the outer
// half row J that the main thread of row J leaves unset, in parallel with
// the main warps (the box schemes of Eqs. em_r_open_bx and em_r_open_bt),
// so that the warp of row J does not run the interior and the boundary
// formulas one after the other.  c: the context of the main thread (k, J).
// ---------------------------------------------------------------------------
template <class R, int M, int RB>
QDS_HD bool outer_active(const MarchCtx<R, M, RB, 0> &c) {
  return !c.closed && c.J >= c.rb0 && c.J < c.rb0 + RB;
}

// phase 1: B_x at n+1/2 on row J, face L-1
template <class R, int M, int RB>
QDS_HD void outer_p1(const MarchCtx<R, M, RB, 0> &c, int L) {
  constexpr int PL = M * RB;
  const int j = c.J, k = c.k;
  if (L < c.xa || L > c.xb + 1) return;
  if (j < c.r0 - 2 || j >= c.r1 + 2) return;
  const int f = L - 1;
  if (!c.face_ok(f)) return;  // the main thread wrote the held-zero face
  const C<R> *a = c.rc[1], *b = c.rc[0];
  const C<R> rp = a[0] + b[0], rm = a[PL] + b[PL], qp = a[2 * PL] + b[2 * PL], qm = a[3 * PL] + b[3 * PL];
  const C<R> er = R(0.25) * (rp + rm), eth = R(0.25) * (qp + qm);
  const C<R> b0 = a[5 * PL];
  const C<R> jtf = c.face_avg(c.jt, k, f, j);
  const C<R> bx = leap_outer<R>(a, b, PL, j, k, c.dr, c.h, c.ih, c.idr, jtf, er, eth, b0);
  c.ex[1][PL] = bx;
  if (c.ax) c.af[1][0] = R(0.5) * (b0 + bx);
  if (c.owned(f, j)) c.store(BX, f, c.gcol(f), bx);
}

// phase 3: T_r+- at n+1 on row J, cell L-1; returns false if a stored value
// is not finite
template <class R, int M, int RB>
QDS_HD bool outer_p3(const MarchCtx<R, M, RB, 0> &c, int L) {
  constexpr int PL = M * RB;
  const int j = c.J;
  if (L < c.xa + 1 || L > c.xb + 1) return true;
  if (j < c.r0 - 1 || j >= c.r1 + 1) return true;
  const int cc = L - 1;
  const C<R> *A = c.rc[2], *B = c.rc[1], *Cn = c.rc[0];
  Shift<R> sh;
  sh.tp = sh.tm = zero<R>();
  if (c.cell_ok(cc)) {
    CurCaller<R, M, RB> cur{c};
    em_shift<R, M, RB, 0>(c, cc, CellsRing<R, PL>{A, B, Cn}, c.ex[2], c.ex[1], cur, sh);
  }
  if (c.ax) {
    C<R> *cs = c.cc[1];
    cs[0] = B[0] + sh.tp;
    cs[PL] = B[PL] + sh.tm;
  }
  if (c.owned(cc, j)) {
    const unsigned gw = c.gcol(cc);
    c.store(TRP, cc, gw, sh.tp);
    c.store(TRM, cc, gw, sh.tm);
    return finite_c(sh.tp);
  }
  return true;
}

// ---------------------------------------------------------------------------
// K2 phase 1: A' (E_x1, B_x1) at face L-1 on rows [r0-1, r1+1), driven by
// j_a,x (and j_a,theta on the outer half row) of that face.
// ---------------------------------------------------------------------------
template <class R, int M, int RB>
QDS_HD void k2_p1(const MarchCtx<R, M, RB, 1> &c, int L) {
  const int j = c.j; constexpr int PL = M * RB;
  if (L < c.xa || L > c.xb) return;
  if (j < c.r0 - 1 || j >= c.r1 + 1 || j < 0 || j >= c.nr) return;
  const int f = L - 1;
  C<R> *ex = c.ex[1];
  const bool own = c.owned(f, j);
  const unsigned gw = own ? c.gcol(f) : 0u;
  if (!c.face_ok(f)) {
    ex[0] = zero<R>();
    ex[PL] = zero<R>();
    if (own) {
      c.store(EX1, f, gw, zero<R>());
      c.store(BX1, f, gw, zero<R>());
    }
    return;
  }
  const C<R> *a = c.rc[1], *b = c.rc[0];
  Leap<R> o;
  em_leap<R, M, RB, 1>(c, a, b, a[6 * PL], a[8 * PL], o);
  ex[0] = o.ex;
  ex[PL] = o.bx;
  if (own) {
    c.store(EX1, f, gw, o.ex);
    c.store(BX1, f, gw, o.bx);
  }
}

// The own-row values of one old column that K2's shift reads after the
// column has left the 4-slot ring: T1 of the cell (and of the row below, and
// all four T1 planes, on the outer half row), and j_a of the face.
template <class R>
struct K2Hist {
  C<R> trp, trm, ttp, ttm, trp1, trm1, jx, jr, jt, jr1;
};

// Cells cc-1 (ha), cc (hb) from the history, cc+1 from the ring.
template <class R, int PL>
struct CellsHist {
  const K2Hist<R> &ha, &hb;
  const C<R> *Cc;
  static QDS_HD C<R> pick(const K2Hist<R> &h, int p, int dj) {
    if (dj == 0) return p == 0 ? h.trp : p == 1 ? h.trm : p == 2 ? h.ttp : h.ttm;
    return p == 0 ? h.trp1 : h.trm1;
  }
  QDS_HD C<R> a(int p, int dj) const { return pick(ha, p, dj); }
  QDS_HD C<R> b(int p, int dj) const { return pick(hb, p, dj); }
  QDS_HD C<R> n(int p, int dj) const { return Cc[p * PL + dj]; }
};

// j_a of faces cc-1 (ha) and cc (hb) from the history.
template <class R>
struct CurHist {
  const K2Hist<R> &ha, &hb;
  int cc, j;
  QDS_HD C<R> jx(int w, int) const { return (w == cc ? hb : ha).jx; }
  QDS_HD C<R> jr(int w, int jj) const {
    const K2Hist<R> &h = w == cc ? hb : ha;
    return jj == j ? h.jr : h.jr1;
  }
  QDS_HD C<R> jt(int w, int) const { return (w == cc ? hb : ha).jt; }
};

// K2 phase 2: C' (T1) at cell L-2 on the owned rows, then the history moves
// on by one column (column L-1 is read before its slot is refilled).
// h[0]: column L-3, h[1]: column L-2.
template <class R, int M, int RB>
QDS_HD void k2_p2(const MarchCtx<R, M, RB, 1> &c, int L, K2Hist<R> (&h)[2], bool &bad) {
  constexpr int PL = M * RB;
  const int j = c.j, k = c.k;
  if (j < c.r0 || j >= c.r1 || j < 0 || j >= c.nr) return;
  if (L >= c.xa + 2 && L <= c.xb + 1) {
    const int cc = L - 2;
    Shift<R> sh;
    CurHist<R> cur{h[0], h[1], cc, j};
    em_shift<R, M, RB, 1>(c, cc, CellsHist<R, PL>{h[0], h[1], c.rc[1]}, c.ex[3], c.ex[2], cur, sh);
    const unsigned gw = c.gcol(cc);
    c.store(TRP1, cc, gw, sh.tp);
    c.store(TRM1, cc, gw, sh.tm);
    c.store(TTP1, cc, gw, sh.up);
    c.store(TTM1, cc, gw, sh.um);
    bad = bad || !finite_c(sh.tp);
  }
  h[0] = h[1];
  if (L > c.L0) {
    const C<R> *p = c.rc[1];
    h[1].trp = p[0];
    h[1].trm = p[PL];
    h[1].ttp = p[2 * PL];
    h[1].ttm = p[3 * PL];
    h[1].jx = p[6 * PL];
    h[1].jr = p[7 * PL];
    h[1].jt = p[8 * PL];
    if (j == c.J) {
      h[1].trp1 = p[-1];
      h[1].trm1 = p[PL - 1];
      h[1].jr1 = p[7 * PL - 1];
    }
  }
}

// Column coordinate of window column cc for the bulk copy: its storage slot,
// or nx (outside the tensor: read as zeros) outside the window.
QDS_HD int march_coord(int cc, int nx, int s, bool per) {
  if (per) { cc %= nx; if (cc < 0) cc += nx; return cc; }
  if (cc < 0 || cc >= nx) return nx;
  const int q = cc + s;
  return q >= nx ? q - nx : q;
}

// Iterations and loaded columns of a CTA with owned columns [xa, xb):
//   K1: columns xa-1 .. xb+1, iterations xa-1 .. xb+2;
//   K2: columns xa-1 .. xb,   iterations xa-1 .. xb+1.
QDS_HD int march_first(int xa) { return xa - 1; }
QDS_HD int march_last(int kind, int xb) { return kind == 0 ? xb + 2 : xb + 1; }
QDS_HD int march_last_col(int kind, int xb) { return kind == 0 ? xb + 1 : xb; }

// Set up the context of thread tid of a CTA (shared by the kernels and the
// host emulation).
template <class R, int M, int RB, int KIND>
QDS_HD void march_ctx(MarchCtx<R, M, RB, KIND> &c, const Inst<R> &I, const MarchItem &it, C<R> *sm,
                      unsigned long long nstep, int tid) {
  c.nx = I.nx; c.nr = I.nr; c.J = I.nr - 1; c.ld = I.ld;
  c.per = (I.flags & F_X_PERIODIC) != 0;
  c.closed = (I.flags & F_R_CLOSED) != 0;
  c.mw = (I.flags & F_MOVING_WINDOW) != 0;
  c.ax = (I.flags & (F_AXION | F_AREM)) != 0;
  c.s = c.mw ? (int)(nstep % (unsigned long long)I.nx) : 0;
  c.P = plane_elems(M, I.nx, I.ld);
  c.h = I.h; c.dr = I.dr; c.ih = I.inv_h; c.idr = I.inv_dr;
  c.ma2 = I.ma2; c.gs = I.gs; c.gj = I.gj;
  const int par = (int)(nstep & 1ull);
  c.o = I.state[par];
  c.n = I.state[par ^ 1];
  c.scr = I.scratch;
  c.P32 = (unsigned)c.P;
  c.ld32 = (unsigned)I.ld;
  c.rb0 = it.rb0; c.r0 = it.r0; c.r1 = it.r1; c.xa = it.xa; c.xb = it.xb;
  c.L0 = march_first(it.xa);
  c.sm = sm;
  c.k = tid / RB;
  c.lr = tid - c.k * RB;
  c.j = it.rb0 + c.lr;
  c.koff = c.k * RB;
  c.off_t = c.koff + c.lr;
  c.gk = (unsigned)c.k * (unsigned)I.nx * (unsigned)I.ld + (unsigned)c.j;
  c.irj = c.j > 0 ? R(1) / (R(c.j) * c.dr) : R(0);
  c.irh = R(1) / ((R(c.j) + R(0.5)) * c.dr);
  c.kirj = R(c.k) * c.irj;
  c.kirh = R(c.k) * c.irh;
}

#if defined(__CUDACC__) && !defined(QDS_EMU)
// ---------------------------------------------------------------------------
// Device: mbarriers and bulk tensor copies (inline PTX).
// ---------------------------------------------------------------------------
__device__ __forceinline__ uint32_t smem_addr(const void *p) { return (uint32_t)__cvta_generic_to_shared(p); }

__device__ __forceinline__ void mbar_init(uint64_t *bar, unsigned count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_addr(bar)), "r"(count) : "memory");
}
__device__ __forceinline__ void mbar_expect_tx(uint64_t *bar, unsigned bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_addr(bar)), "r"(bytes) : "memory");
}
__device__ __forceinline__ bool mbar_try_wait(uint64_t *bar, unsigned parity) {
  uint32_t ok;
  asm volatile(
      "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}\n"
      : "=r"(ok)
      : "r"(smem_addr(bar)), "r"(parity)
      : "memory");
  return ok != 0;
}
// bounded wait: false if the phase did not complete within the limit
__device__ __forceinline__ bool mbar_wait(uint64_t *bar, unsigned parity) {
  for (int it = 0; it < (1 << 20); it++)
    if (mbar_try_wait(bar, parity)) return true;
  return false;
}
__device__ __forceinline__ void tma_load_4d(void *dst, const CUtensorMap *map, int c0, int c1, int c2, int c3,
                                            uint64_t *bar) {
  asm volatile(
      "cp.async.bulk.tensor.4d.shared::cluster.global.tile.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3, %4, %5}], [%6];"
      ::"r"(smem_addr(dst)), "l"(reinterpret_cast<uint64_t>(map)), "r"(c0), "r"(c1), "r"(c2), "r"(c3),
        "r"(smem_addr(bar))
      : "memory");
}

// Tensor maps of one instance: the old state as [field][mode][column][row]
// boxes for K1 (fields TRP..TAM) and K2 (TRP1..BX1), per ping-pong half,
// and the j_a scratch planes.
struct MarchMaps {
  CUtensorMap k1[2];
  CUtensorMap k2[2];
  CUtensorMap ja;
};

template <class R, int M, int KIND>
__device__ __forceinline__ void march_issue(const MarchMaps &mm, int par, C<R> *slot_ptr, int row0, int coord,
                                            uint64_t *bar, unsigned bytes, int RB) {
  asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
  mbar_expect_tx(bar, bytes);
  const int r0c = sizeof(R) == 4 ? row0 : 2 * row0;  // FP64: two 8-byte words per complex
  if (KIND == 0) {
    tma_load_4d(slot_ptr, &mm.k1[par], r0c, coord, 0, 0, bar);
  } else {
    tma_load_4d(slot_ptr, &mm.k2[par], r0c, coord, 0, TRP1, bar);
    tma_load_4d(slot_ptr + 6 * M * RB, &mm.ja, r0c, coord, 0, 1, bar);
  }
}

// The step kernel of one mode count and ring height (KIND 0: K1, 1: K2): one
// CTA per work item, M * RB threads.
// K1 has one more warp, the boundary warp (outer_p1 / outer_p3).
template <int M, int RB, int KIND>
constexpr int march_threads() { return M * RB + (KIND == 0 ? 32 : 0); }

template <class R, int M, int RB, int KIND>
__global__ void __launch_bounds__(march_threads<M, RB, KIND>(), KIND == 1 ? 2 : 1) march_kernel(const Inst<R> *__restrict__ insts,
                                                       const MarchMaps *__restrict__ maps,
                                                       const MarchItem *__restrict__ items, Ctrl *ctrl) {
  using Sh = MarchShape<R, M, RB, KIND>;
  extern __shared__ __align__(128) unsigned char smraw[];
  const MarchItem it = items[blockIdx.x];
  const Inst<R> &I = insts[it.inst];
  const unsigned long long nstep = ctrl->step;
  const int par = (int)(nstep & 1ull);
  const int tid = threadIdx.x;
  C<R> *sm = reinterpret_cast<C<R> *>(smraw);
  // the boundary warp's lane k takes the context of the main thread (k, J)
  constexpr int NMAIN = M * RB;
  const bool bwarp = tid >= NMAIN;
  const int bk = tid - NMAIN;
  const int ctid = bwarp ? bk * RB + min(max(I.nr - 1 - it.rb0, 0), RB - 1) : tid;
  MarchCtx<R, M, RB, KIND> c;
  march_ctx<R, M, RB, KIND>(c, I, it, sm, nstep, bwarp && bk < M ? ctid : (bwarp ? 0 : tid));
  bool bact = false;
  if constexpr (KIND == 0) bact = bwarp && bk < M && outer_active<R, M, RB>(c);
  c.jx = step_src(I.jx, I, ctrl);
  c.jr = step_src(I.jr, I, ctrl);
  c.jt = step_src(I.jt, I, ctrl);
  c.sext = step_src(I.sext, I, ctrl);
  c.in_rp = step_inflow(I.in_rp, I, ctrl);
  c.in_tm = step_inflow(I.in_tm, I, ctrl);
  constexpr int NS = Sh::NS;
  constexpr int BAR = ((KIND == 0 ? Sh::O_ST + Sh::PL : Sh::O_AF) * (int)sizeof(C<R>) + 15) / 16 * 16;
  uint64_t *bar = reinterpret_cast<uint64_t *>(smraw + BAR);
  const bool ar = (I.flags & F_AREM) != 0;
  if (tid == 0) {
    for (int b = 0; b < NS; b++) mbar_init(&bar[b], 1);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  __syncthreads();
  const int L0 = c.L0, L1 = march_last(KIND, it.xb), C1 = march_last_col(KIND, it.xb);
  constexpr unsigned bytes = (unsigned)(kPlanes * Sh::PL * sizeof(C<R>));
  const MarchMaps &mm = maps[it.inst];
  auto issue = [&](int col) {
    const int s2 = (col - L0) % NS;
    march_issue<R, M, KIND>(mm, par, sm + s2 * Sh::SS, it.rb0, march_coord(col, c.nx, c.s, c.per), &bar[s2], bytes,
                            RB);
  };
  // (test hook: with bit 0 of ctrl->test set the first column is never
  // fetched, so that its bounded wait runs out)
  const bool withhold = (ctrl->test & 1u) != 0;
  if (tid == 0)
    for (int col = L0; col <= C1 && col < L0 + 3; col++)
      if (!(withhold && col == L0)) issue(col);
  K1Regs<R> rg;
  rg.gam_prev = rg.gam = rg.tap_prev = rg.tam_prev = zero<R>();
  rg.bad = false;
  K2Hist<R> hist[2];
  if constexpr (KIND == 1) {
    const C<R> z = zero<R>();
    for (int q = 0; q < 2; q++) hist[q] = K2Hist<R>{z, z, z, z, z, z, z, z, z, z};
  }
  for (int L = L0; L <= L1; L++) {
    c.iter(L);
    // column L (if any) has landed; a copy that did not complete within the
    // limit sets the error flag, the CTA lets its copies in flight land and
    // stops (the failure is agreed at the barrier that ends the phase)
    const bool ok = L > C1 || mbar_wait(&bar[(L - L0) % NS], (unsigned)(((L - L0) / NS) & 1));
    if (ok) {
      if constexpr (KIND == 0) {
        if (!bwarp) k1_inflow<R, M, RB>(c, L);
        if (!bwarp) k1_p1<R, M, RB>(c, L);
        else if (bact) outer_p1<R, M, RB>(c, L);
      } else {
        k2_p1<R, M, RB>(c, L);
      }
    }
    if (__syncthreads_or(!ok)) {
      if (tid == 0) {
        atomicOr(&ctrl->err, kErrTimeout);
        for (int col = L; col <= C1 && col < L + 3; col++)
          if (!(withhold && col == L0)) mbar_wait(&bar[(col - L0) % NS], (unsigned)(((col - L0) / NS) & 1));
      }
      __syncthreads();
      return;
    }
    if constexpr (KIND == 0) {
      if (!bwarp) k1_p2<R, M, RB>(c, L, ar);
      __syncthreads();
      if (!bwarp) k1_p3<R, M, RB>(c, L, rg);
      else if (bact && !outer_p3<R, M, RB>(c, L)) rg.bad = true;
    } else {
      k2_p2<R, M, RB>(c, L, hist, rg.bad);
    }
    __syncthreads();
    // the ring slot of column L-2 (K1) / L-1 (K2, its values now in the
    // history registers) is no longer read
    if (tid == 0 && L + 3 <= C1) issue(L + 3);
  }
  if (__syncthreads_or(rg.bad) && tid == 0) atomicOr(&ctrl->err, kErrNonfinite);
}
#endif

}  // namespace qds
