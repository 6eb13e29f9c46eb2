// qds_adjoint.cuh -- the transpose of one QDS EM + axion step.
//
// For a real functional L of the complex state, the adjoint of a complex
// value z is zb = dL/dRe z + i dL/dIm z; a term y = c x (c complex) gives
// xb += conj(c) yb, and y = conj(x) gives xb += conj(yb).  The regenerated
// group never feeds back into the EM fields or the axion (Sec. 2.2, reading
// of the step order), so the adjoint of an axion-energy functional has no
// regenerated part and this transpose covers the EM group and the axion.
//
// Adjoint fields live in the canonical window-order layout (no ring offset)
// in the working precision.  The forward state of the step (time n) is read
// through a Tile (its row stride and ring offset).  Every entry of the old
// adjoint is written once by the thread that owns it (a gather: no atomic
// scatters), in three passes over the (x, r) points:
//   AD_SRC   faces: the old T_a and Gamma_a's adjoint from the new T_a and
//            phi (Eqs. Ta_plus_update, Ta_minus_update, phi_update), d L / d g,
//            and the transpose of the bilinear source S_a (Eq.
//            mode_convolution) at the forward state, kept per face;
//   AD_LEAP  faces: the total adjoints of E_x, B_x^(n+1/2) (new state, the T
//            shift's face sources, the source means), the old E_x, B_x (Eqs.
//            Ex_update, axis_Ex, Phix_explicit, em_r_open_bx), phi and
//            phi_prev (Gamma_a's Laplacian and mass with the outer ghost);
//   AD_CELL  cells: the old T (shifted copies, Eqs. Trp/Trm/Ttp/Ttm_update,
//            axis_Ttheta; the outer boxes, Eq. em_r_open_bt; the leapfrog
//            and source-mean terms of the two neighbouring faces).
// The transpose of the +x shift is the -x shift and vice versa; the window
// shift reads the new state's adjoint one column over.  Open x, open r,
// optional moving window; no periodic or closed test modes.
#pragma once

#include "qds_stages.cuh"

namespace qds {

enum AdStage { AD_SRC = 0, AD_LEAP, AD_CELL, N_ADSTAGE };

// scratch planes of the adjoint (window order), each M*nx*nr, on faces:
// Gamma_a's adjoint; the adjoints of the face means of the axion source
// (eX, bX, rp, rm, qp, qm); the total adjoints of E_x, B_x^(n+1/2)
enum AdScr { SB_G = 0, SB_EXB, SB_BXB, SB_RPB, SB_RMB, SB_QPB, SB_QMB, SB_EXT, SB_BXT, N_SB };

template <class R, int M>
struct Adj {
  Tile<R, M, false> f;  // forward state at time n
  const C<R> *fnext;    // forward state at the end of the step, same layout (null: recompute E_x, B_x^(n+1/2))
  const C<R> *ln;       // adjoint of the state after the step (canonical layout)
  C<R> *lo;             // adjoint of the state before the step (canonical layout)
  C<R> *sb;             // scratch planes (N_SB)
  double *dg;           // accumulated dL/dg (null: not wanted)
  int nx, nr, J;
  unsigned P;           // elements of one field's plane set, M * nx * nr (< 2^32: checked at create)
  bool mw;
  bool zero_regen;      // also write the (zero) regenerated planes of lo
  R h, dr, ih, idr;
  R gs, ma2;
  R c_kab, c_ikab, c_irJ;  // (a - b)/(a + b), 1/(a + b) of the outer box, 1/r_J (set with set_consts)

  QDS_HD void set_consts() {
    c_kab = kab();
    c_ikab = R(1) / (ka() + kb());
    c_irJ = R(1) / (R(J) * dr);
  }

  // Rows passed to the accessors below are inside the box (callers guard
  // the radial neighbours); columns are checked.
  // the radial neighbours, held inside the box (used under guards that
  // exclude the axis and the last row: the clamp only keeps a hoisted load
  // inside the buffer)
  QDS_HD int up(int j) const { return j < J ? j + 1 : J; }
  QDS_HD int dn(int j) const { return j > 0 ? j - 1 : 0; }
  // 32-bit signed element offsets (one instance's state has fewer than 2^31
  // elements).  A load that the compiler hoists above its guard must still
  // address the buffer: the guarded accessors clamp their indices, and a
  // signed offset keeps any other stray index next to the buffer.
  QDS_HD int ai(int field, int k, int w, int j) const { return field * (int)P + k * (nx * nr) + w * nr + j; }
  QDS_HD bool in_cell(int w) const { return w >= 0 && w < nx; }
  QDS_HD bool in_face(int w) const { return w >= 0 && w <= nx - 2; }
  // adjoint of the new state in the fixed box (before the window shift)
  QDS_HD C<R> lnew(int field, int k, int w, int j) const {
    if (mw) w -= 1;
    const bool ok = w >= 0 && w < nx;
    const int wc = ok ? w : 0;
    chk(field, NFIELD, k, wc, j, "adjoint read of the new state's adjoint");
    const C<R> v = ldg(ln + ai(field, k, wc, j));
    return ok ? v : zero<R>();
  }
  QDS_HD C<R> lnew_prev(int k, int w) const {
    if (mw) w -= 1;
    const bool ok = w >= 0 && w < nx;
    const int wc = ok ? w : 0;
    chk(0, 1, k, wc, 0, "adjoint phi_prev read");
    const C<R> v = ldg(ln + ((int)NFIELD * (int)P + k * nx + wc));
    return ok ? v : zero<R>();
  }
#if defined(QDS_EMU)
  QDS_HD void chk(int field, int nf, int k, int w, int j, const char *what) const {
    QDS_CHECK(field >= 0 && field < nf && k >= 0 && k < M && w >= 0 && w < nx && j >= 0 && j < nr, what);
  }
#else
  QDS_HD void chk(int, int, int, int, int, const char *) const {}
#endif
  QDS_HD C<R> &old(int field, int k, int w, int j) const { chk(field, NFIELD, k, w, j, "adjoint store"); return lo[ai(field, k, w, j)]; }
  QDS_HD C<R> &oldprev(int k, int w) const { chk(0, 1, k, w, 0, "adjoint phi_prev store"); return lo[(int)NFIELD * (int)P + k * nx + w]; }
  QDS_HD C<R> &s(int plane, int k, int w, int j) const { chk(plane, N_SB, k, w, j, "adjoint scratch"); return sb[ai(plane, k, w, j)]; }
  // reads of scratch planes that the running pass does not write
  QDS_HD C<R> sr(int plane, int k, int w, int j) const { chk(plane, N_SB, k, w, j, "adjoint scratch read"); return ldg(sb + ai(plane, k, w, j)); }
  // scratch on a face, zero off the faces and rows of the box
  QDS_HD C<R> sf(int plane, int k, int w, int j) const {
    const bool ok = in_face(w) && j >= 0 && j < nr;
    const C<R> v = sr(plane, k, ok ? w : 0, ok ? j : 0);
    return ok ? v : zero<R>();
  }
  // adjoint of the new T (q = 0..3: T_r^+, T_r^-, T_th^+, T_th^-) at cell c
  QDS_HD C<R> tn(int q, int k, int c, int j) const {
    return in_cell(c) ? lnew(TRP + q, k, c, j) : zero<R>();
  }
  // adjoints of the new T_a^+- at cell c, with the phi update's share
  // (phi^(n+1) at the faces on either side takes (h/4) T_a^(n+1/2) of c)
  QDS_HD C<R> phi_share(int k, int c, int j) const {
    C<R> pl = in_face(c - 1) ? lnew(PHI, k, c - 1, j) : zero<R>();
    C<R> pr = in_face(c) ? lnew(PHI, k, c, j) : zero<R>();
    return (R(0.25) * h) * (pl + pr);
  }
  QDS_HD C<R> tap_n(int k, int c, int j) const {
    return in_cell(c) ? lnew(TAP, k, c, j) + phi_share(k, c, j) : zero<R>();
  }
  QDS_HD C<R> tam_n(int k, int c, int j) const {
    return in_cell(c) ? lnew(TAM, k, c, j) + phi_share(k, c, j) : zero<R>();
  }
  // box-scheme weights of the outer half row (Eqs. em_r_open_bx/bt)
  QDS_HD R ka() const { return R(0.5) * ih; }
  QDS_HD R kb() const { return R(0.5) * idr; }
  QDS_HD R kab() const { return (ka() - kb()) / (ka() + kb()); }
  // adjoint of B_th^(n+1) on the last half row at cell c (zero off the box)
  QDS_HD C<R> box_bt(int k, int c) const { return tn(0, k, c, J) - tn(1, k, c, J); }
  // effective adjoints of the new T at cell c: T_r on half row J-1 with the
  // fold of the outer box, T_th on the axis only for m = 1 (axis_Ttheta)
  QDS_HD C<R> trp_e(int k, int c, int j) const {
    if (!in_cell(c)) return zero<R>();
    C<R> v = tn(0, k, c, j);
    if (j == J - 1) v += (R(-0.5) * c_kab) * box_bt(k, c);
    return v;
  }
  QDS_HD C<R> trm_e(int k, int c, int j) const {
    if (!in_cell(c)) return zero<R>();
    C<R> v = tn(1, k, c, j);
    if (j == J - 1) v -= (R(-0.5) * c_kab) * box_bt(k, c);
    return v;
  }
  QDS_HD C<R> tt_e(int q, int k, int c, int j) const {
    if (!in_cell(c) || (j == 0 && k != 1)) return zero<R>();
    return tn(q, k, c, j);
  }
};

// Transpose of the mode convolution C_m{A, B} (Eq. mode_convolution) for all
// output modes at once: Ab += dC/dA^T Sb, Bb += dC/dB^T Sb (scaled by wgt).
template <class R, int M>
QDS_HD void conv_T(const C<R> *A, const C<R> *B, const C<R> *Sb, R wgt, C<R> *Ab, C<R> *Bb) {
  // m = 0: A0 B0 + (1/2) sum_k Re(A_k conj B_k)
  {
    C<R> s0 = wgt * Sb[0];
    Ab[0] += mul_cj(s0, B[0]);
    Bb[0] += mul_cj(s0, A[0]);
    #pragma unroll
    for (int k = 1; k < M; k++) {
      Ab[k] += (R(0.5) * s0.re) * B[k];
      Bb[k] += (R(0.5) * s0.re) * A[k];
    }
  }
  #pragma unroll
  for (int m = 1; m < M; m++) {
    C<R> t = (R(0.5) * wgt) * Sb[m];
    #pragma unroll
    for (int k = 0; k <= m && k < M; k++) {  // A_k B_l, k + l = m
      int l = m - k;
      if (l < M) {
        Ab[k] += mul_cj(t, B[l]);
        Bb[l] += mul_cj(t, A[k]);
      }
    }
    #pragma unroll
    for (int l = 0; l + m < M; l++) {  // A_{l+m} conj(B_l)
      Ab[l + m] += B[l] * t;
      Bb[l] += mul_cj(A[l + m], t);
    }
    #pragma unroll
    for (int k = 0; k + m < M; k++) {  // conj(A_k) B_{k+m}
      Ab[k] += mul_cj(B[k + m], t);
      Bb[k + m] += A[k] * t;
    }
  }
}

// ---------------------------------------------------------------------------
// Per-thread views for one mode: the columns a point reads, resolved once
// (window shift, column checks, clamped base), so that each read is an
// offset from a base and a select.  Rows passed are inside the box.
//
// The new state's adjoint at the cells c + dc, dc = -1, 0, +1.
template <class R, int M>
struct NewCols {
  const C<R> *p[3];
  bool ok[3];
  int P;
#if defined(QDS_EMU)
  const Adj<R, M> *ad;
  int k, c;
#endif
  QDS_HD NewCols(const Adj<R, M> &a, int k_, int c_) {
    P = (int)a.P;
    const int shift = a.mw ? 1 : 0;
#pragma unroll
    for (int d = 0; d < 3; d++) {
      const int w = c_ + d - 1, ws = w - shift;
      ok[d] = a.in_cell(w) && ws >= 0 && ws < a.nx;
      p[d] = a.ln + (k_ * (a.nx * a.nr) + (ok[d] ? ws : 0) * a.nr);
    }
#if defined(QDS_EMU)
    ad = &a;
    k = k_;
    c = c_;
#endif
  }
  QDS_HD C<R> at(int field, int dc, int row) const {
#if defined(QDS_EMU)
    ad->chk(field, NFIELD, k, 0, row, "adjoint read of the new state's adjoint (column view)");
#endif
    const C<R> v = ldg(p[dc + 1] + (field * P + row));
    return ok[dc + 1] ? v : zero<R>();
  }
};

// The scratch planes at the faces c - 1 (df = 0) and c (df = 1).
template <class R, int M>
struct ScrFaces {
  const C<R> *p[2];
  bool ok[2];
  int P;
#if defined(QDS_EMU)
  const Adj<R, M> *ad;
  int k;
#endif
  QDS_HD ScrFaces(const Adj<R, M> &a, int k_, int c) {
    P = (int)a.P;
#pragma unroll
    for (int d = 0; d < 2; d++) {
      const int f = c - 1 + d;
      ok[d] = a.in_face(f);
      p[d] = a.sb + (k_ * (a.nx * a.nr) + (ok[d] ? f : 0) * a.nr);
    }
#if defined(QDS_EMU)
    ad = &a;
    k = k_;
#endif
  }
  QDS_HD C<R> at(int plane, int df, int row) const {
#if defined(QDS_EMU)
    ad->chk(plane, N_SB, k, 0, row, "adjoint scratch read (face view)");
#endif
    const C<R> v = ldg(p[df] + (plane * P + row));
    return ok[df] ? v : zero<R>();
  }
};

// ---------------------------------------------------------------------------
// The E_x and B_x^(n+1/2) adjoints that the T shift's face sources give at
// face f, row j (Eqs. Trp/Trm/Ttp/Ttm_update; axis rules of Sec. 2.3; on the
// last row, E_r^(n+1) takes Gamma_r of the faces on either side).
template <class R, int M>
QDS_HD void unshift_face(const Adj<R, M> &a, const NewCols<R, M> &nc, int k, int j, C<R> &ex, C<R> &bx) {
  const int J = a.J;
  const R h = a.h, dr = a.dr, idr = a.idr, kf = R(-0.5) * a.c_kab;
  const int jm = j > 0 ? j - 1 : 0, jp = j < J ? j + 1 : J;
  // effective new T at cell f + dc (the box fold of T_r on half row J - 1,
  // T_th on the axis only for m = 1)
  auto boxbt = [&](int dc) { return nc.at(TRP, dc, J) - nc.at(TRM, dc, J); };
  auto trp = [&](int dc, int jj) {
    C<R> v = nc.at(TRP, dc, jj);
    if (jj == J - 1) v += kf * boxbt(dc);
    return v;
  };
  auto trm = [&](int dc, int jj) {
    C<R> v = nc.at(TRM, dc, jj);
    if (jj == J - 1) v -= kf * boxbt(dc);
    return v;
  };
  auto tt = [&](int q, int dc, int jj) { return (jj == 0 && k != 1) ? zero<R>() : nc.at(TRP + q, dc, jj); };
  // T_r sources of half rows j and j - 1, T_th sources of rows j, j + 1, 0
  const C<R> sp_j = h * trp(1, j), sm_j = h * trm(0, j);
  const C<R> Gr = sp_j + sm_j, Pr = sp_j - sm_j;
  const C<R> sp_m = h * trp(1, jm), sm_m = h * trm(0, jm);
  const C<R> Pr_m = sp_m - sm_m;
  const C<R> tp_j = h * tt(2, 0, j), tm_j = h * tt(3, 1, j);
  const C<R> Gt = tp_j + tm_j, Pt = tp_j - tm_j;
  const C<R> tp_p = h * tt(2, 0, jp), tm_p = h * tt(3, 1, jp);
  const C<R> Gt_p = tp_p + tm_p;
  const C<R> tp_0 = h * tt(2, 0, 0), tm_0 = h * tt(3, 1, 0);
  const C<R> Gt_0 = tp_0 + tm_0, Pt_0 = tp_0 - tm_0;
  ex = zero<R>();
  bx = zero<R>();
  // E_x(f, j) enters Phi_r of half rows j and j-1 and Phi_th of row j
  if (j < J) ex -= idr * Pr;
  if (j >= 1) {
    ex += idr * Pr_m;
    ex += imul(-R(k) / (R(j) * dr), Pt);
  }
  if (k == 1 && j <= 1) ex += imul(j == 1 ? -idr : idr, Pt_0);  // axis: Phi_th = i (E_x(1) - E_x(0)) / dr
  // B_x(f, j) enters Gamma_r of half row j and Gamma_th of rows j, j+1
  const R irh = R(1) / ((R(j) + R(0.5)) * dr);
  if (j < J) bx += imul(R(k) * irh, Gr);
  else {
    const C<R> Gb = (R(0.5) * h) * (nc.at(TRP, 1, J) + nc.at(TRM, 1, J) + nc.at(TRP, 0, J) + nc.at(TRM, 0, J));
    bx += imul(R(k) * irh, Gb);
  }
  if (j >= 1) bx -= idr * Gt;
  else if (k == 1) bx += (-R(2) * idr) * Gt_0;
  if (j + 1 <= J) bx += idr * Gt_p;
}

// The forward state around face f as the source transpose reads it: the
// columns f and f + 1 only (cells f, f + 1; face f), rows inside the box
// (the leapfrog helpers guard their radial neighbours).  Each column's
// ring slot is resolved once; the interface is the Tile's, for the forward
// helpers ex_update, bx_interior and bx_outer.
template <class R, int M>
struct AdjFwd {
  using Real = R;
  const C<R> *c0, *c1;  // columns f and f + 1 of field 0, mode 0
  const C<R> *n0;       // column f of the state at the end of the step (null: none)
  const C<R> *jx, *jt, *sext;
  unsigned P, kst;      // field and mode strides of the working planes
  int f, nx, nr, J;
  R h, dr, ih, idr;
  QDS_HD AdjFwd(const Tile<R, M, false> &t, const C<R> *next, bool mw, int f_) {
    f = f_; nx = t.nx; nr = t.nr; J = t.J;
    h = t.h; dr = t.dr; ih = t.ih; idr = t.idr;
    jx = t.jx; jt = t.jt; sext = t.sext;
    P = (unsigned)t.P;
    kst = (unsigned)(t.nx * t.ld);
    int s0 = f + t.s, s1 = f + 1 + t.s;  // ring slots (f + 1 <= nx - 1)
    if (s0 >= nx) s0 -= nx;
    if (s1 >= nx) s1 -= nx;
    c0 = t.o + (unsigned)(s0 * t.ld);
    c1 = t.o + (unsigned)(s1 * t.ld);
    // the window shift moves no data (ring offset): face f of the step's
    // fixed box is the same ring slot in the next state, except the rear
    // column, which the shift clears for the new front column
    n0 = (next && !(mw && f == 0)) ? next + (unsigned)(s0 * t.ld) : nullptr;
#if defined(QDS_EMU)
    o = t.o;
    len = t.state_len;
#endif
  }
#if defined(QDS_EMU)
  const C<R> *o;
  size_t len;
#endif
  QDS_HD C<R> cell(int field, int k, int w, int j) const {
    // rows outside the box are never read (the leapfrog helpers guard
    // them); the clamp only keeps a hoisted load inside the buffer
    const int jc = j < 0 ? 0 : (j > J ? J : j);
    const C<R> *p = (w == f ? c0 : c1) + ((int)field * (int)P + k * (int)kst + jc);
#if defined(QDS_EMU)
    QDS_CHECK((w == f || w == f + 1) && j >= 0 && j < nr && (size_t)(p - o) < len, "adjoint forward read");
#endif
    return ldg(p);
  }
  QDS_HD C<R> face(int field, int k, int w, int j) const { return cell(field, k, w, j); }
  // E_x, B_x^(n+1/2) at face f as the step stored them
  QDS_HD C<R> next_face(int field, int k, int j) const {
    const int jc = j > J ? J : j;
    return ldg(n0 + ((int)field * (int)P + k * (int)kst + jc));
  }
  QDS_HD C<R> Er(int grp, int k, int w, int j) const { return R(0.5) * (cell(grp + TRP, k, w, j) + cell(grp + TRM, k, w, j)); }
  QDS_HD C<R> Bt(int grp, int k, int w, int j) const { return R(0.5) * (cell(grp + TRP, k, w, j) - cell(grp + TRM, k, w, j)); }
  QDS_HD C<R> Et(int grp, int k, int w, int j) const { return R(0.5) * (cell(grp + TTP, k, w, j) + cell(grp + TTM, k, w, j)); }
  QDS_HD C<R> Br(int grp, int k, int w, int j) const { return R(0.5) * (cell(grp + TTP, k, w, j) - cell(grp + TTM, k, w, j)); }
  // caller's sources [M][nx][nr] in window order
  QDS_HD C<R> srcv(const C<R> *a, int k, int w, int j) const {
    if (!a) return zero<R>();
    const int jc = j < 0 ? 0 : (j > J ? J : j);
    return ldg(a + ((k * nx + w) * nr + jc));
  }
};

// AD_SRC, face (f, j): Gamma_a's adjoint from the new T_a (Eqs. Ta_plus/
// Ta_minus_update with the phi update's share), d L / d g, and the transpose
// of the bilinear source S_a (Eq. mode_convolution) at the forward state:
// the adjoints of its six face means, kept per face for the next stages.
template <class R, int M>
QDS_HD void adj_src(const Adj<R, M> &a, int f, int j, double &dg_acc) {
  if (!a.in_face(f)) {
    // the ends of the T_a shifts: T_a^+ of the last cell and T_a^- of the
    // first feed no new T_a
    #pragma unroll
    for (int k = 0; k < M; k++) {
      a.old(TAP, k, f, j) = zero<R>();
      a.old(TAM, k, 0, j) = zero<R>();
    }
    return;
  }
  const int J = a.J;
  const bool top = (j == J);
  const R h = a.h;
  const AdjFwd<R, M> t(a.f, a.fnext, a.mw, f);
  C<R> Gb[M], Sb[M];
  const bool last_face = f + 1 > a.nx - 2;  // phi of cell f + 1 is off the faces
  #pragma unroll
  for (int k = 0; k < M; k++) {
    // T_a^+(c + 1) = T_a^+(c) + h Gamma_a(c + 1/2), T_a^-(c) = T_a^-(c + 1) + h
    // Gamma_a(c + 1/2): face f gives the old T_a^+ of cell f and T_a^- of f + 1;
    // the new T_a adjoints carry the phi update's share of the faces on
    // either side of their cell
    const NewCols<R, M> nc(a, k, f);
    const C<R> ph0 = nc.at(PHI, 0, j);
    const C<R> ph1 = last_face ? zero<R>() : nc.at(PHI, 1, j);
    const C<R> tp = nc.at(TAP, 1, j) + (R(0.25) * h) * (ph0 + ph1);
    const C<R> tm = nc.at(TAM, 0, j) + (R(0.25) * h) * (nc.at(PHI, -1, j) + ph0);
    a.old(TAP, k, f, j) = tp;
    a.old(TAM, k, f + 1, j) = tm;
    Gb[k] = h * (tp + tm);
    Sb[k] = a.gs * Gb[k];
    a.s(SB_G, k, f, j) = Gb[k];
  }
  // S = C{eX, bX} + (1/2)(C{rp, qp} - C{rm, qm}) at the forward state
  C<R> eX[M], bX[M], rp[M], rm[M], qp[M], qm[M];
  #pragma unroll
  for (int k = 0; k < M; k++) {
    C<R> exn, bxn, exn1;
    if (t.n0) {  // the leapfrog's results, as the step stored them
      exn = t.next_face(EX, k, j);
      bxn = t.next_face(BX, k, j);
      exn1 = top ? exn : t.next_face(EX, k, j + 1);
    } else {     // recomputed (Eqs. Ex_update, Phix_explicit, em_r_open_bx)
      exn = ex_update(t, 0, k, f, j, t.srcv(t.jx, k, f, j));
      bxn = (j < J) ? bx_interior(t, 0, k, f, j)
                    : bx_outer(t, 0, k, f, R(0.5) * (t.srcv(t.jt, k, f, j) + t.srcv(t.jt, k, f + 1, j)),
                               bx_interior(t, 0, k, f, j - 1));
      exn1 = top ? exn : ex_update(t, 0, k, f, j + 1, t.srcv(t.jx, k, f, j + 1));
    }
    const C<R> eo = t.face(EX, k, f, j), eo1 = top ? eo : t.face(EX, k, f, j + 1);
    eX[k] = R(0.25) * (eo + eo1 + exn + exn1);
    bX[k] = R(0.5) * (t.face(BX, k, f, j) + bxn);
    const int j1 = top ? j : j + 1;
    rp[k] = R(0.5) * (t.cell(TRP, k, f, j) + t.cell(TRP, k, f + 1, j));
    rm[k] = R(0.5) * (t.cell(TRM, k, f, j) + t.cell(TRM, k, f + 1, j));
    qp[k] = R(0.25) * (t.cell(TTP, k, f, j) + t.cell(TTP, k, f + 1, j) + t.cell(TTP, k, f, j1) + t.cell(TTP, k, f + 1, j1));
    qm[k] = R(0.25) * (t.cell(TTM, k, f, j) + t.cell(TTM, k, f + 1, j) + t.cell(TTM, k, f, j1) + t.cell(TTM, k, f + 1, j1));
  }
  if (a.dg) {  // Gamma_a depends on g through g S (physical variables)
    // the point's share in the working precision (FP64 arithmetic is slow on
    // this part), the sums over points in FP64
    R acc = R(0);
    #pragma unroll
    for (int m = 0; m < M; m++) {
      C<R> S = conv<R, M>(m, eX, bX) + R(0.5) * (conv<R, M>(m, rp, qp) - conv<R, M>(m, rm, qm));
      S += t.srcv(t.sext, m, f, j);
      acc += Gb[m].re * S.re + Gb[m].im * S.im;
    }
    dg_acc += (double)acc;  // the caller reduces and adds to *a.dg
  }
  C<R> eXb[M], bXb[M], rpb[M], rmb[M], qpb[M], qmb[M];
  #pragma unroll
  for (int k = 0; k < M; k++) eXb[k] = bXb[k] = rpb[k] = rmb[k] = qpb[k] = qmb[k] = zero<R>();
  conv_T<R, M>(eX, bX, Sb, R(1), eXb, bXb);
  conv_T<R, M>(rp, qp, Sb, R(0.5), rpb, qpb);
  conv_T<R, M>(rm, qm, Sb, R(-0.5), rmb, qmb);
  #pragma unroll
  for (int k = 0; k < M; k++) {
    a.s(SB_EXB, k, f, j) = eXb[k];
    a.s(SB_BXB, k, f, j) = bXb[k];
    a.s(SB_RPB, k, f, j) = rpb[k];
    a.s(SB_RMB, k, f, j) = rmb[k];
    a.s(SB_QPB, k, f, j) = qpb[k];
    a.s(SB_QMB, k, f, j) = qmb[k];
  }
}

// AD_LEAP, face (f, j): the total adjoints of E_x and B_x^(n+1/2) (the new
// state's, the T shift's face sources', the source means') and from them the
// old E_x, B_x (Eqs. Ex_update, axis_Ex, Phix_explicit, em_r_open_bx).
template <class R>
struct LeapOut {
  C<R> ex, bx;    // the old E_x, B_x adjoints
  C<R> ext, bxt;  // the total E_x, B_x^(n+1/2) adjoints (faces only)
  C<R> ph, prev;  // the old phi and (last row) phi_prev adjoints
};

template <class R, int M>
QDS_HD LeapOut<R> leap_vals(const Adj<R, M> &a, int k, int f, int j) {
  const int J = a.J;
  LeapOut<R> o;
  o.ex = o.bx = o.ext = o.bxt = o.ph = o.prev = zero<R>();
  if (!a.in_face(f)) return o;
  const R kab = a.c_kab, dr = a.dr, ih = a.ih;
  const int jm = j > 0 ? j - 1 : 0, jp = j < J ? j + 1 : J;
  const NewCols<R, M> nf(a, k, f);  // dc = 0: cell f, +1: cell f + 1
  const C<R> *sp = a.sb + (k * (a.nx * a.nr) + f * a.nr);
  const int P = (int)a.P;
  auto S = [&](int plane, int row) {
#if defined(QDS_EMU)
    a.chk(plane, N_SB, k, f, row, "adjoint scratch read (own face)");
#endif
    return ldg(sp + (plane * P + row));
  };
  // ---- phi: carried over by the phi update, Gamma_a's Laplacian and mass
  // with the outer ghost (-(2 dr/h) phi(J) + phi(J-1)), phi_prev (phi off
  // the faces, in the last column, has no adjoint: the zeros above) ----
  {
    C<R> ph = nf.at(PHI, 0, j);
    if (j == J) ph += a.lnew_prev(k, f);
    // d_i = 1 / ((i + 1/2) dr^2) = idr / r_(i+1/2)
    const R irh = R(1) / ((R(j) + R(0.5)) * dr);
    const R den = irh * a.idr;
    R cc = -(R(2 * j + 1)) * den - (R(k * k) * irh * irh + a.ma2);
    if (j == J) cc += R(J + 1) * den * (-R(2) * dr * ih);
    ph += cc * S(SB_G, j);
    if (j >= 1) ph += (R(j) * (a.idr / ((R(j) - R(0.5)) * dr))) * S(SB_G, jm);
    if (j + 1 <= J) {
      const int i = j + 1;
      const R di = a.idr / ((R(i) + R(0.5)) * dr);
      R w = R(i) * di;
      if (i == J) w += R(J + 1) * di;
      ph += w * S(SB_G, jp);
    }
    o.ph = ph;
    if (j == J) o.prev = (R(J + 1) * den * R(2) * dr * ih) * S(SB_G, J);
  }
  // eX(f, jj) is the mean of E_x at rows jj and jj + 1 (jj on the last row)
  // of the old and the new E_x: row j takes eX of rows j and j - 1
  const C<R> exb_m = j >= 1 ? S(SB_EXB, jm) : zero<R>();
  const C<R> e4 = R(0.25) * ((j == J ? R(2) : R(1)) * S(SB_EXB, j) + exb_m);
  C<R> ex, bx;
  unshift_face(a, nf, k, j, ex, bx);
  const C<R> ext = nf.at(EX, 0, j) + ex + e4;
  C<R> bxt = nf.at(BX, 0, j) + bx + R(0.5) * S(SB_BXB, j);
  C<R> bxJ = zero<R>();  // the last row's, for the box of row J - 1
  if (j == J - 1) {
    C<R> exJ, bxJs;
    unshift_face(a, nf, k, J, exJ, bxJs);
    bxJ = nf.at(BX, 0, J) + bxJs + R(0.5) * S(SB_BXB, J);
    bxt -= kab * bxJ;  // the box reads B_x^(n+1/2)(J - 1)
  }
  o.ext = ext;
  o.bxt = bxt;
  // E_x^(n+1/2) = E_x^(n-1/2) + h Gamma_x; on the axis only m = 0 moves
  o.ex = ((j > 0 || k == 0) ? ext : zero<R>()) + e4;
  // B_x: interior rows carry it over; the box of the last row weighs
  // B_x(J) by (a - b)/(a + b) and B_x(J - 1) by 1
  C<R> ob = R(0.5) * S(SB_BXB, j);
  if (j < J) ob += bxt;
  else ob += kab * bxt;
  if (j == J - 1) ob += bxJ;
  o.bx = ob;
  return o;
}

template <class R, int M>
QDS_HD void leap_store(const Adj<R, M> &a, int k, int f, int j, const LeapOut<R> &o) {
  a.old(EX, k, f, j) = o.ex;
  a.old(BX, k, f, j) = o.bx;
  a.old(PHI, k, f, j) = o.ph;
  if (j == a.J) a.oldprev(k, f) = o.prev;
  if (a.in_face(f)) {
    a.s(SB_EXT, k, f, j) = o.ext;
    a.s(SB_BXT, k, f, j) = o.bxt;
  }
}

// AD_CELL, cell (c, j): the old T, T_a, phi and phi_prev, gathered from the
// new state's adjoint (shifted copies), the outer boxes of the cells c - 1 ..
// c + 1, and the face adjoints of faces c - 1 and c (source means, E_x, B_x).
template <class R>
struct CellOut {
  C<R> t[4];      // the old T_r^+, T_r^-, T_th^+, T_th^-
};

template <class R, int M>
QDS_HD CellOut<R> cell_vals(const Adj<R, M> &a, int k, int c, int j) {
  CellOut<R> o;
  const int J = a.J;
  const R h = a.h, dr = a.dr, idr = a.idr, ih = a.ih;
  const R kab = a.c_kab, ikab = a.c_ikab, irJ = a.c_irJ, kf = R(-0.5) * kab;
  const int jm = j > 0 ? j - 1 : 0, jp = j < J ? j + 1 : J;
  const NewCols<R, M> nc(a, k, c);  // cells c - 1, c, c + 1
  const ScrFaces<R, M> sf(a, k, c);  // faces c - 1, c
  // reciprocal radii of the rows this cell's faces reach (0 where unused)
  const R ir_j = j >= 1 ? R(1) / (R(j) * dr) : R(0);                // 1/r_j
  const R ir_j1 = R(1) / (R(j + 1) * dr);                           // 1/r_(j+1)
  const R ir_hm = j >= 1 ? R(1) / ((R(j) - R(0.5)) * dr) : R(0);    // 1/r_(j-1/2)
  const R ir_h = R(1) / ((R(j) + R(0.5)) * dr);                     // 1/r_(j+1/2)
  auto boxbt = [&](int dc) { return nc.at(TRP, dc, J) - nc.at(TRM, dc, J); };
  C<R> trp = zero<R>(), trm = zero<R>(), ttp = zero<R>(), ttm = zero<R>();
  // the transverse fields map to T^+- as E_r, B_th -> T_r and E_th, B_r -> T_th
  auto Er = [&](C<R> v) { trp += R(0.5) * v; trm += R(0.5) * v; };
  auto Bt = [&](C<R> v) { trp += R(0.5) * v; trm -= R(0.5) * v; };
  auto Et = [&](C<R> v) { ttp += R(0.5) * v; ttm += R(0.5) * v; };
  auto Br = [&](C<R> v) { ttp += R(0.5) * v; ttm -= R(0.5) * v; };
  // ---- the shifted copies (-x for T_r^+, T_th^-, +x for T_r^-, T_th^+) ----
  if (j < J) {
    trp += nc.at(TRP, 1, j);
    trm += nc.at(TRM, -1, j);
    if (j == J - 1) {  // the fold of the outer box into half row J - 1
      trp += kf * boxbt(1);
      trm -= kf * boxbt(-1);
    }
  } else {  // last half row: E_r^(n+1)(c') takes (T_r^+(c'-1) + T_r^-(c'+1))/2
    trp += R(0.5) * (nc.at(TRP, 1, J) + nc.at(TRM, 1, J));
    trm += R(0.5) * (nc.at(TRP, -1, J) + nc.at(TRM, -1, J));
  }
  if (j > 0 || k == 1) {  // T_th on the axis only for m = 1
    ttp += nc.at(TTP, -1, j);
    ttm += nc.at(TTM, 1, j);
  }
  // ---- the outer T_r boxes of cells c - 1, c, c + 1 (Eq. em_r_open_bt) ----
  if (j >= J - 1) {
    // B_th^(n+1) = (R - (a-b) B_th^(n+1)(J-1) + (a-b) B_th(J) + (a+b) B_th(J-1)) / (a+b),
    // R = -(1/4) ih (E_r(c+1) - E_r(c-1)) - (1/(2 rJ)) (B_th + i m B_r) + ...
    const C<R> Bb = boxbt(0);
    const C<R> Rb = ikab * Bb;
    const C<R> er_m = (R(-0.125) * ih) * (ikab * boxbt(-1));  // from cell c - 1
    const C<R> er_p = (R(-0.125) * ih) * (ikab * boxbt(1));   // from cell c + 1
    if (j == J) {
      Bt(kab * Bb + (R(-0.25) * irJ) * Rb);
      Br(imul(R(k) * R(0.5) * irJ, Rb));
    } else {
      Bt(Bb + (R(-0.25) * irJ) * Rb);
    }
    Er(er_m - er_p);
  }
  // ---- faces c - 1 and c (a face off the box reads as zero) ----
  const R tw = (j == J) ? R(2) : R(1);
#pragma unroll
  for (int df = 0; df < 2; df++) {
    // the source means: rp, rm on row j; qp, qm on rows j, j + 1 (j, j on the last)
    trp += R(0.5) * sf.at(SB_RPB, df, j);
    trm += R(0.5) * sf.at(SB_RMB, df, j);
    C<R> qpm = tw * sf.at(SB_QPB, df, j), qmm = tw * sf.at(SB_QMB, df, j);
    if (j >= 1) {
      qpm += sf.at(SB_QPB, df, jm);
      qmm += sf.at(SB_QMB, df, jm);
    }
    ttp += R(0.25) * qpm;
    ttm += R(0.25) * qmm;
    // E_x leapfrog (Eq. Ex_update; axis_Ex for m = 0)
    if (j == 0 && k == 0) Bt((h * R(2) * idr) * sf.at(SB_EXT, df, 0));
    if (j >= 1) {
      const C<R> eb = sf.at(SB_EXT, df, j);
      Bt((R(0.5) * h * (R(j) + R(0.5)) * ir_j) * eb);
      Br(imul(R(-0.5) * h * R(k) * ir_j, eb));
    }
    if (j + 1 <= J) Bt((R(-0.5) * h * (R(j) + R(0.5)) * ir_j1) * sf.at(SB_EXT, df, jp));
    // B_x leapfrog (Eq. Phix_explicit) on rows j - 1, j; the box of row J
    if (j >= 1) Et((R(-0.5) * h * R(j) * ir_hm) * sf.at(SB_BXT, df, jm));
    if (j < J) {
      const C<R> bb = sf.at(SB_BXT, df, j);
      Et((R(0.5) * h * R(j) * ir_h) * bb);
      Er(imul(R(0.5) * h * R(k) * ir_h, bb));
    }
    if (j >= J - 1) {
      // B_x(J) = (R - (a-b) B_x^(n+1/2)(J-1) + (a-b) B_x(J) + (a+b) B_x(J-1)) / (a+b),
      // R = (1/2) ih (B_r(f+1, J) - B_r(f, J)) - (1/(2 rJ)) (E_th + i m E_r) - ...
      const C<R> Rb = ikab * sf.at(SB_BXT, df, J);
      if (j == J) {
        Br((df == 0 ? R(0.5) : R(-0.5)) * ih * Rb);  // face c - 1 reads B_r(c) with +, face c with -
        Et((R(-0.25) * irJ) * Rb);
      }
      Er(imul(R(k) * R(0.125) * irJ, Rb));
    }
  }
  o.t[0] = trp;
  o.t[1] = trm;
  o.t[2] = ttp;
  o.t[3] = ttm;
  return o;
}

template <class R, int M>
QDS_HD void cell_store(const Adj<R, M> &a, int k, int c, int j, const CellOut<R> &o) {
#pragma unroll
  for (int q = 0; q < 4; q++) a.old(TRP + q, k, c, j) = o.t[q];
  if (a.zero_regen)
    for (int fl = TRP1; fl < NFIELD; fl++) a.old(fl, k, c, j) = zero<R>();
}

// One point of a pass: AD_SRC covers every mode of face w (the source
// couples the modes); AD_LEAP and AD_CELL one mode k.
template <class R, int M>
QDS_HD void adj_point(const Adj<R, M> &a, int st, int k, int w, int j, double &dg_acc) {
  if (st == AD_SRC) adj_src<R, M>(a, w, j, dg_acc);
  else if (st == AD_LEAP) leap_store<R, M>(a, k, w, j, leap_vals<R, M>(a, k, w, j));
  else cell_store<R, M>(a, k, w, j, cell_vals<R, M>(a, k, w, j));
}

}  // namespace qds
