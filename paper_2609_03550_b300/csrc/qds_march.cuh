// qds_march.cuh -- the x-marching step kernels.
//
// One CTA owns a band of radial rows [r0, r1) of one instance, all retained
// modes, and a segment of window columns [xa, xb); it walks the segment
// along +x one column per iteration.  Each new column of the old state (all
// fields the kernel reads, all modes, the band and its radial halo) arrives
// in a ring of shared-memory slots by one bulk tensor copy (TMA) completed on
// an mbarrier, two columns ahead of the column being computed.  Columns
// outside the window and rows outside the grid are filled with zeros by the
// copy itself (out-of-range coordinates), which is the open boundary of
// Eqs. em_x_open / axion_x_open; the moving window is the copy's column
// coordinate (the ring offset), not a data move.
//
// The stages of one step are column-lagged, all operands in shared memory,
// and arranged in two phases per column so that each phase is spread evenly
// over all threads and one barrier separates the phases.  Iteration L
// (column L has arrived):
//   K1 (EM field + axion + axion current):
//     phase 1:  A  E_x, B_x to n+1/2 at face L-1   (Eqs. Ex_update, Phix_explicit)
//               D  j_a at face L-3 -> scratch       (Eqs. jax/jar/jat_mode)
//     phase 2:  per (row, mode), one thread:
//               B  Gamma_a of that mode at face L-1 (Eqs. source_mode_*, mode_convolution)
//               C  T^(n+1), T_a^(n+1/2) at cell L-1 (Eqs. Trp/Trm/Ttp/Ttm_update,
//                  Ta_plus/minus_update; needs Gamma_a of faces L-2, L-1 of the
//                  same row and mode, formed by the same thread)
//               P  phi^(n+1) at face L-2            (Eq. phi_update)
//   K2 (axion-regenerated EM, driven by j_a), one phase:
//               A' E_x1, B_x1 to n+1/2 at face L-1, C' T1^(n+1) at cell L-2.
// The point formulas are those of qds_stages.cuh, read through MarchTile.
// The state is read once and written once per step (K1: 9 planes, K2: 6
// planes and the 3 j_a planes read back), each value of a column stored by
// the thread of its (row, mode) in one coalesced pass.
#pragma once

#include "qds_stages.cuh"

#if defined(__CUDACC__) && !defined(QDS_EMU)
#include <cuda.h>

#include "qds_kernels.cuh"
#endif

namespace qds {

constexpr int kRing = 6;       // ring slots: columns L-3 .. L live, two in flight
constexpr int kHalo1 = 4;      // K1 radial halo (three rows needed, kept even)
constexpr int kHalo2 = 2;      // K2 radial halo
constexpr int kNF = 9;         // planes per ring slot (K1: 9 fields; K2: 6 fields + 3 j_a planes)

// One CTA's work: instance, output rows [r0, r1), smem row base rb0,
// output columns [xa, xb).
struct MarchItem {
  int inst, r0, r1, rb0, xa, xb, pad0, pad1;
};

// Shared-memory plan of a march launch (elements of C<R>).
struct MarchGeo {
  int RB;        // rows per slot (band + halo, even)
  int slot;      // elements per ring slot (rounded to 128 bytes)
  int off_a, off_g, off_t, off_p, off_bar;  // intermediate planes, mbarriers (bytes for off_bar)
  int bytes;     // dynamic shared memory
};

template <class R>
QDS_HD MarchGeo march_geo(int kind, int M, int RB) {
  MarchGeo g;
  g.RB = RB;
  const int per128 = 128 / (int)sizeof(C<R>);
  g.slot = (kNF * M * RB + per128 - 1) / per128 * per128;
  int o = kRing * g.slot;
  g.off_a = o; o += 4 * 2 * M * RB;              // E_x, B_x (group of the kernel) at n+1/2, four faces
  g.off_g = o; if (kind == 0) o += 2 * M * RB;  // Gamma_a, two faces
  g.off_t = o; if (kind == 0) o += 2 * 6 * M * RB;  // T^(n+1), T_a^(n+1/2), two cells
  g.off_p = o; if (kind == 0) o += M * RB;      // phi^(n+1), one face
  int b = o * (int)sizeof(C<R>);
  b = (b + 15) / 16 * 16;
  g.off_bar = b;
  g.bytes = b + kRing * 8;
  return g;
}

// Shared-memory view of one CTA's step (the accessor of qds_stages.cuh).
// KIND 0: ring planes are the fields TRP..TAM; KIND 1: the fields
// TRP1..BX1, then j_a,x, j_a,r, j_a,theta.  Coordinates: lx is the window
// column (x0 = 0), lr the row (r0 = 0).
template <class R, int M, int KIND>
struct MarchTile {
  using Real = R;
  static constexpr int kM = M;
  static constexpr bool kSM = true;  // intermediates are the CTA's planes
  static constexpr int FB = KIND == 0 ? 0 : TRP1;  // first field of the ring
  const C<R> *jx, *jr, *jt, *sext;
  R gs, gj, ma2;
  uint32_t flags;
  int nx, nr, J, ld;
  int x0, r0;          // accessor origin: always 0
  int s;               // ring offset of the window
  bool per, closed, mw;
  size_t P;
  const C<R> *o;       // old state (global): phi_prev only
  C<R> *n;             // new state (global)
  C<R> *scr;           // scratch planes (global): j_a written by K1
  R h, dr, ih, idr;
  C<R> *ring, *sa, *sg, *st, *sp;  // shared memory
  int RB, rb0, SS;     // rows per plane, first row, elements per ring slot
  int xa, xb, b_r0, b_r1;  // owned columns and rows
#if defined(QDS_EMU)
  int sm_len;
#endif

  QDS_HD bool cell_ok(int w) const { return per || (w >= 0 && w < nx); }
  QDS_HD bool face_ok(int w) const { return per || (w >= 0 && w <= nx - 2); }
  QDS_HD void set_point(int) const {}
  // storage slot of window column w (inside the window)
  QDS_HD int slot(int w) const {
    if (per) { w %= nx; if (w < 0) w += nx; return w; }
    int q = w + s;
    return q >= nx ? q - nx : q;
  }
  QDS_HD int ri(int fi, int k, int w, int j) const {
    const int i = ((w + 4 * kRing) % kRing) * SS + (fi * M + k) * RB + (j - rb0);
#if defined(QDS_EMU)
    QDS_CHECK(j - rb0 >= 0 && j - rb0 < RB && fi >= 0 && fi < kNF && w >= -4 * kRing, "march ring index");
#endif
    return i;
  }
  QDS_HD C<R> cell(int field, int k, int w, int j) const { return ring[ri(field - FB, k, w, j)]; }
  QDS_HD C<R> face(int field, int k, int w, int j) const {
    if (!per && w == nx - 1) return zero<R>();  // the held-zero face
    return ring[ri(field - FB, k, w, j)];
  }
  QDS_HD C<R> prev(int k, int w) const {
    if (!face_ok(w)) return zero<R>();
    return ldg(o + (size_t)NFIELD * P + (size_t)k * nx + slot(w));
  }
  QDS_HD C<R> srcv(const C<R> *a, int k, int w, int j) const {
    if (!a || !cell_ok(w) || j < 0 || j >= nr) return zero<R>();
    if (per) { w %= nx; if (w < 0) w += nx; }
    return ldg(a + ((size_t)k * nx + w) * nr + j);
  }
  QDS_HD bool owned(int w, int j) const { return w >= xa && w < xb && j >= b_r0 && j < b_r1; }
  QDS_HD void store(int field, int k, int w, int j, C<R> v) const {
    if (mw && w == 0) v = zero<R>();  // the rear column becomes the new front
    n[(size_t)field * P + ((size_t)k * nx + slot(w)) * ld + j] = v;
  }
  QDS_HD void store_prev(int k, int w, C<R> v) const {
    if (mw && w == 0) v = zero<R>();
    n[(size_t)NFIELD * P + (size_t)k * nx + slot(w)] = v;
  }
  QDS_HD C<R> Er(int grp, int k, int w, int j) const { return R(0.5) * (cell(grp + TRP, k, w, j) + cell(grp + TRM, k, w, j)); }
  QDS_HD C<R> Bt(int grp, int k, int w, int j) const { return R(0.5) * (cell(grp + TRP, k, w, j) - cell(grp + TRM, k, w, j)); }
  QDS_HD C<R> Et(int grp, int k, int w, int j) const { return R(0.5) * (cell(grp + TTP, k, w, j) + cell(grp + TTM, k, w, j)); }
  QDS_HD C<R> Br(int grp, int k, int w, int j) const { return R(0.5) * (cell(grp + TTP, k, w, j) - cell(grp + TTM, k, w, j)); }

  QDS_HD int pi(int slot2, int pl, int npl, int k, int j) const {
    const int i = ((slot2 * npl + pl) * M + k) * RB + (j - rb0);
#if defined(QDS_EMU)
    QDS_CHECK(j - rb0 >= 0 && j - rb0 < RB, "march plane row");
#endif
    return i;
  }
  // E_x, B_x at n+1/2 of the kernel's group at face lx (four faces kept)
  QDS_HD C<R> &sA(int pl, int k, int lx, int lr) const { return sa[pi(lx & 3, pl, 2, k, lr)]; }
  QDS_HD C<R> &sG(int k, int lx, int lr) const { return sg[pi(lx & 1, 0, 1, k, lr)]; }
  QDS_HD C<R> &sT(int pl, int k, int lx, int lr) const { return st[pi(lx & 1, pl, 6, k, lr)]; }
  QDS_HD C<R> &sP(int k, int lx, int lr) const { return sp[pi(0, 0, 1, k, lr)]; }
  // KIND 0: j_a (pl 2..4) into the scratch planes; KIND 1: pl 0, 1 the
  // regenerated E_x1, B_x1 at n+1/2, pl 2..4 the j_a planes of the ring
  QDS_HD C<R> &sJ(int pl, int k, int lx, int lr) const {
    if (KIND == 0) return scr[(size_t)(pl - 1) * P + ((size_t)k * nx + slot(lx)) * ld + lr];
    if (pl < 2) return sa[pi(lx & 3, pl, 2, k, lr)];
    return ring[ri(6 + pl - 2, k, lx, lr)];
  }
};

// ---------------------------------------------------------------------------
// Stages (every thread of the CTA calls each one; the kernel puts a barrier
// between the phases).  Rows are clipped to [0, nr).
// ---------------------------------------------------------------------------
QDS_HD int clip_lo(int a) { return a < 0 ? 0 : a; }

// K1 A: E_x, B_x at face w on rows [r0-2, r1+2); one (row, mode) per thread.
template <class R, int M>
QDS_HD void m1_leap(const MarchTile<R, M, 0> &t, int w, int tid, int nth) {
  const int lo = clip_lo(t.b_r0 - 2), hi = t.b_r1 + 2 < t.nr ? t.b_r1 + 2 : t.nr, nrow = hi - lo;
  if (nrow <= 0) return;
  const bool fok = t.face_ok(w);
  for (int q = tid; q < M * nrow; q += nth) {
    const int k = q / nrow, j = lo + (q - k * nrow);
    C<R> ex = zero<R>(), bx = zero<R>();
    if (fok) {
      C<R> jtf = zero<R>();
      if (j == t.J && !t.closed) jtf = R(0.5) * (t.srcv(t.jt, k, w, j) + t.srcv(t.jt, k, w + 1, j));
      leap_point(t, 0, k, w, j, t.srcv(t.jx, k, w, j), jtf, ex, bx);
    }
    t.sA(0, k, w, j) = ex;
    t.sA(1, k, w, j) = bx;
    if (t.owned(w, j)) { t.store(EX, k, w, j, ex); t.store(BX, k, w, j, bx); }
  }
}

// K1 B, C, P for one (row, mode) per thread on rows [r0-1, r1+1): Gamma_a of
// that mode at face wb (if do_b), then T, T_a at cell wb (if do_c, reading
// Gamma_a of faces wb-1, wb of the same row and mode), then phi at face wb-1
// on rows [r0-1, r1) (if do_p) from T_a of cells wb-1 (previous column, same
// thread) and wb.  Returns true if a stored T_r^+ or T_a^+ is not finite.
template <class R, int M>
QDS_HD bool m1_source_shift(const MarchTile<R, M, 0> &t, int wb, bool do_b, bool do_c, bool do_p, bool ax, int tid,
                            int nth) {
  const int lo = clip_lo(t.b_r0 - 1), hi = t.b_r1 + 1 < t.nr ? t.b_r1 + 1 : t.nr, nrow = hi - lo;
  bool bad = false;
  if (nrow <= 0) return bad;
  Faces0<MarchTile<R, M, 0>> fs{t};
  const int c = wb;
  const bool live = t.cell_ok(c);
  for (int q = tid; q < M * nrow; q += nth) {
    const int k = q / nrow, j = lo + (q - k * nrow);
    if (ax && do_b) source_point(t, wb, j, TileLeapVals<MarchTile<R, M, 0>>{t, wb, j}, k);
    C<R> ap = zero<R>(), am = zero<R>();
    if (do_c) {
      C<R> tp = zero<R>(), tm = zero<R>(), up = zero<R>(), um = zero<R>();
      if (live) {
        if (j < t.J || t.closed) tr_interior(t, fs, 0, k, c, j, tp, tm);
        else {
          C<R> ip, im_;
          tr_interior(t, fs, 0, k, c, j - 1, ip, im_);
          tr_outer(t, fs, 0, k, c, R(0.5) * (ip - im_), j, tp, tm);
        }
        tt_update(t, fs, 0, k, c, j, up, um);
        if (ax) {
          ap = t.cell(TAP, k, c - 1, j) + t.h * t.sG(k, c - 1, j);
          am = t.cell(TAM, k, c + 1, j) + t.h * t.sG(k, c, j);
        }
      }
      t.sT(0, k, c, j) = tp; t.sT(1, k, c, j) = tm;
      t.sT(2, k, c, j) = up; t.sT(3, k, c, j) = um;
      if (ax) { t.sT(4, k, c, j) = ap; t.sT(5, k, c, j) = am; }
      if (t.owned(c, j)) {
        t.store(TRP, k, c, j, tp); t.store(TRM, k, c, j, tm);
        t.store(TTP, k, c, j, up); t.store(TTM, k, c, j, um);
        if (ax) { t.store(TAP, k, c, j, ap); t.store(TAM, k, c, j, am); }
        bad = bad || !finite_c(tp) || !finite_c(ap);
      }
    }
    if (ax && do_p && j < t.b_r1) {
      const int w = c - 1;
      C<R> v = zero<R>();
      const C<R> po = t.face(PHI, k, w, j);
      if (t.face_ok(w)) v = po + (R(0.25) * t.h) * (am + t.sT(5, k, w, j) + ap + t.sT(4, k, w, j));
      t.sP(k, w, j) = v;
      if (t.owned(w, j)) {
        t.store(PHI, k, w, j, v);
        if (j == t.J) t.store_prev(k, w, po);
      }
    }
  }
  return bad;
}

// K1 D: j_a at face w on the owned rows, into the scratch planes; the three
// components are spread over the threads.
template <class R, int M>
QDS_HD void m1_current(const MarchTile<R, M, 0> &t, int w, int tid, int nth) {
  const int lo = t.b_r0, hi = t.b_r1, nrow = hi - lo;
  if (w < t.xa || w >= t.xb) return;
  constexpr int NC = M < 3 ? M : 3;
  for (int q = tid; q < NC * nrow; q += nth) {
    const int cq = q / nrow, j = lo + (q - cq * nrow);
    const int comp = NC == 1 ? 7 : NC == 2 ? (cq == 0 ? 3 : 4) : (1 << cq);
    C<R> jax[M], jat[M];
    current_point(t, w, j, jax, jat, TileNewVals<MarchTile<R, M, 0>>{t, w}, comp);
  }
}

// K2 A': E_x1, B_x1 at face w on rows [r0-1, r1+1).
template <class R, int M>
QDS_HD void m2_leap(const MarchTile<R, M, 1> &t, int w, int tid, int nth) {
  const int lo = clip_lo(t.b_r0 - 1), hi = t.b_r1 + 1 < t.nr ? t.b_r1 + 1 : t.nr, nrow = hi - lo;
  if (nrow <= 0) return;
  const bool fok = t.face_ok(w);
  for (int q = tid; q < M * nrow; q += nth) {
    const int k = q / nrow, j = lo + (q - k * nrow);
    C<R> ex = zero<R>(), bx = zero<R>();
    if (fok) leap_point(t, TRP1, k, w, j, t.sJ(2, k, w, j), t.sJ(4, k, w, j), ex, bx);
    t.sA(0, k, w, j) = ex;
    t.sA(1, k, w, j) = bx;
    if (t.owned(w, j)) { t.store(EX1, k, w, j, ex); t.store(BX1, k, w, j, bx); }
  }
}

// K2 C': T1 at cell c on the owned rows; true if a stored T_r1^+ is not
// finite.
template <class R, int M>
QDS_HD bool m2_shift(const MarchTile<R, M, 1> &t, int c, int tid, int nth) {
  const int lo = t.b_r0, hi = t.b_r1, nrow = hi - lo;
  bool bad = false;
  if (c < t.xa || c >= t.xb) return bad;
  Faces1<MarchTile<R, M, 1>> fs{t};
  for (int q = tid; q < M * nrow; q += nth) {
    const int k = q / nrow, j = lo + (q - k * nrow);
    C<R> tp, tm, up, um;
    if (j < t.J || t.closed) tr_interior(t, fs, TRP1, k, c, j, tp, tm);
    else {
      C<R> ip, im_;
      tr_interior(t, fs, TRP1, k, c, j - 1, ip, im_);
      tr_outer(t, fs, TRP1, k, c, R(0.5) * (ip - im_), j, tp, tm);
    }
    tt_update(t, fs, TRP1, k, c, j, up, um);
    t.store(TRP1, k, c, j, tp); t.store(TRM1, k, c, j, tm);
    t.store(TTP1, k, c, j, up); t.store(TTM1, k, c, j, um);
    bad = bad || !finite_c(tp);
  }
  return bad;
}

// Columns and iterations of one CTA with output columns [xa, xb).
//   K1: loads xa-1 .. xb+1; iterations xa-1 .. xb+2; A, B at face L-1 for
//       L in [xa, xb+1]; C at cell L-1 for L in [xa+1, xb+1]; P at face L-2
//       for L in [xa+2, xb+1]; D at face L-3 for L in [xa+3, xb+2].
//   K2: loads xa-1 .. xb; iterations xa-1 .. xb+1; A' at face L-1 for L in
//       [xa, xb]; C' at cell L-2 for L in [xa+2, xb+1].
QDS_HD int march_first(int, int xa) { return xa - 1; }
QDS_HD int march_last(int kind, int xb) { return kind == 0 ? xb + 2 : xb + 1; }
QDS_HD int march_last_col(int kind, int xb) { return kind == 0 ? xb + 1 : xb; }

// One iteration's phases, shared by the kernel and the host emulation.
template <class R, int M>
QDS_HD bool m1_phase1(const MarchTile<R, M, 0> &t, int L, bool ar, int tid, int nth) {
  if (L >= t.xa && L <= t.xb + 1) m1_leap<R, M>(t, L - 1, tid, nth);
  if (ar && L >= t.xa + 3) m1_current<R, M>(t, L - 3, tid, nth);
  return false;
}
template <class R, int M>
QDS_HD bool m1_phase2(const MarchTile<R, M, 0> &t, int L, bool ax, int tid, int nth) {
  const bool do_b = L >= t.xa && L <= t.xb + 1;
  const bool do_c = L >= t.xa + 1 && L <= t.xb + 1;
  const bool do_p = L >= t.xa + 2 && L <= t.xb + 1;
  if (!do_b && !do_c && !do_p) return false;
  return m1_source_shift<R, M>(t, L - 1, do_b, do_c, do_p, ax, tid, nth);
}
template <class R, int M>
QDS_HD bool m2_phase(const MarchTile<R, M, 1> &t, int L, int tid, int nth) {
  if (L >= t.xa && L <= t.xb) m2_leap<R, M>(t, L - 1, tid, nth);
  bool bad = false;
  if (L >= t.xa + 2) bad = m2_shift<R, M>(t, L - 2, tid, nth);
  return bad;
}

// Column coordinate of window column c for the bulk copy: its storage slot,
// or nx (outside the tensor: filled with zeros) outside the window.
QDS_HD int march_coord(int c, int nx, int s, bool per) {
  if (per) { c %= nx; if (c < 0) c += nx; return c; }
  if (c < 0 || c >= nx) return nx;
  const int q = c + s;
  return q >= nx ? q - nx : q;
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

// The step kernel of one mode count: one CTA per work item.
template <class R, int M, int KIND>
__global__ void __launch_bounds__(256, 2) march_kernel(const Inst<R> *__restrict__ insts,
                                                    const MarchMaps *__restrict__ maps,
                                                    const MarchItem *__restrict__ items, Ctrl *ctrl, MarchGeo geo) {
  extern __shared__ __align__(128) unsigned char smraw[];
  const MarchItem it = items[blockIdx.x];
  const Inst<R> &I = insts[it.inst];
  const unsigned long long nstep = ctrl->step;
  const int par = (int)(nstep & 1ull);
  MarchTile<R, M, KIND> t;
  t.jx = step_src(I.jx, I, ctrl);
  t.jr = step_src(I.jr, I, ctrl);
  t.jt = step_src(I.jt, I, ctrl);
  t.sext = step_src(I.sext, I, ctrl);
  t.gs = I.gs; t.gj = I.gj; t.ma2 = I.ma2;
  t.flags = I.flags;
  t.nx = I.nx; t.nr = I.nr; t.J = I.nr - 1; t.ld = I.ld;
  t.x0 = 0; t.r0 = 0;
  t.per = (I.flags & F_X_PERIODIC) != 0;
  t.closed = (I.flags & F_R_CLOSED) != 0;
  t.mw = (I.flags & F_MOVING_WINDOW) != 0;
  t.s = t.mw ? (int)(nstep % (unsigned long long)I.nx) : 0;
  t.P = plane_elems(M, I.nx, I.ld);
  t.o = I.state[par];
  t.n = I.state[par ^ 1];
  t.scr = I.scratch;
  t.h = I.h; t.dr = I.dr; t.ih = I.inv_h; t.idr = I.inv_dr;
  C<R> *sm = reinterpret_cast<C<R> *>(smraw);
  t.ring = sm;
  t.sa = sm + geo.off_a;
  t.sg = sm + geo.off_g;
  t.st = sm + geo.off_t;
  t.sp = sm + geo.off_p;
  t.RB = geo.RB;
  t.rb0 = it.rb0;
  t.SS = geo.slot;
  t.xa = it.xa; t.xb = it.xb; t.b_r0 = it.r0; t.b_r1 = it.r1;
  uint64_t *bar = reinterpret_cast<uint64_t *>(smraw + geo.off_bar);
  const int tid = threadIdx.x, nth = blockDim.x;
  const bool ax = (I.flags & (F_AXION | F_AREM)) != 0, ar = (I.flags & F_AREM) != 0;

  // zero the intermediate planes (the first iterations read slots not yet written)
  for (int q = tid; q < (geo.off_bar / (int)sizeof(C<R>)) - geo.off_a; q += nth) sm[geo.off_a + q] = zero<R>();
  if (tid == 0) {
    for (int b = 0; b < kRing; b++) mbar_init(&bar[b], 1);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  __syncthreads();
  const int L0 = march_first(KIND, it.xa), L1 = march_last(KIND, it.xb), C1 = march_last_col(KIND, it.xb);
  const unsigned bytes = (unsigned)(kNF * M * geo.RB * sizeof(C<R>));
  const MarchMaps &mm = maps[it.inst];
  auto issue = [&](int c) {
    const int s2 = (c + 4 * kRing) % kRing;
    march_issue<R, M, KIND>(mm, par, sm + s2 * geo.slot, it.rb0, march_coord(c, t.nx, t.s, t.per), &bar[s2], bytes,
                            geo.RB);
  };
  // (test hook: with bit 0 of ctrl->test set the first column is never
  // fetched, so that its bounded wait runs out)
  const bool withhold = (ctrl->test & 1u) != 0;
  if (tid == 0)
    for (int c = L0; c <= C1 && c < L0 + 3; c++)
      if (!(withhold && c == L0)) issue(c);
  bool bad = false;  // a non-finite value was stored
  for (int L = L0; L <= L1; L++) {
    // column L (if any) has landed; a copy that did not complete within the
    // limit sets the error flag, the CTA lets its copies in flight land and
    // stops (the failure is agreed at the barrier that ends the phase)
    const bool ok = L > C1 || mbar_wait(&bar[(L + 4 * kRing) % kRing], (unsigned)(((L - L0) / kRing) & 1));
    if constexpr (KIND == 0) {
      if (ok) m1_phase1<R, M>(t, L, ar, tid, nth);
    } else {
      if (ok) bad |= m2_phase<R, M>(t, L, tid, nth);
    }
    if (__syncthreads_or(!ok)) {
      if (tid == 0) {
        atomicOr(&ctrl->err, kErrTimeout);
        for (int c = L; c <= C1 && c < L + 3; c++)
          if (!(withhold && c == L0))
            mbar_wait(&bar[(c + 4 * kRing) % kRing], (unsigned)(((c - L0) / kRing) & 1));
      }
      __syncthreads();
      return;
    }
    // column L-3 is no longer read: fetch column L+3 into its slot
    if (tid == 0 && L + 3 <= C1) issue(L + 3);
    if constexpr (KIND == 0) {
      bad |= m1_phase2<R, M>(t, L, ax, tid, nth);
      __syncthreads();
    }
  }
  if (__syncthreads_or(bad) && tid == 0) atomicOr(&ctrl->err, kErrNonfinite);
}
#endif

}  // namespace qds
