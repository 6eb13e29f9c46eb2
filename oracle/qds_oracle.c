/*
 * qds_oracle.c -- plain FP64 CPU oracle of the QDS (quasi-cylindrical
 * direction-splitting) Maxwell + axion field step.
 *
 * TEST INFRASTRUCTURE ONLY.  This file is the slow, obviously-correct
 * restatement of the paper's update equations against which the CUDA path is
 * checked.  Only the tests, the smoke check and the benchmark's CPU-baseline
 * leg may load it.  It shares no code, header or table with the CUDA library.
 *
 * Every field is a complex<double> azimuthal-mode plane (Sec. 2, Eq. fourier
 * decomposition): array[m][i][j] with m the mode, i the x index, j the radial
 * index.  Normalised units c = eps0 = mu0 = hbar = 1, h = dx = c dt.
 *
 * Staggering (Fig. 1 is not available; positions are read off the equation
 * subscripts of Sec. 2.1, 2.2, 2.4):
 *   T_r^{+-}  (i, j+1/2, n)     half row j stored at index j
 *   T_th^{+-} (i, j, n)         integer row j
 *   E_x       (i+1/2, j, n-1/2) face i stored at index i
 *   B_x       (i+1/2, j+1/2, n-1/2)
 *   phi       (i+1/2, j+1/2, n)
 *   T_a^{+-}  (i, j+1/2, n-1/2)
 *   j_x (i+1/2, j, n)   j_r (i, j+1/2, n+1/2)   j_th (i, j, n+1/2)
 * Radii r_j = j dr, r_{j+1/2} = (j+1/2) dr.  Faces 0..nx-2 are real; face
 * nx-1 is held at zero unless x is periodic.
 *
 * Pinned by the tests against the paper and closed forms: exact one-cell
 * transport of k_perp = 0 waves, the electrostatic steady state, the QDS and
 * Klein-Gordon dispersion relations, the theta-quadrature definition of the
 * mode convolution, the vanishing vacuum two-colour source, exact linearity
 * in g, resonant growth, the axion/regenerated-field energy exchange (sign
 * and scale of j_a), and the paper's printed vacuum group velocity.
 *
 * Parity unpinned (no closed form or paper value fixes them; the oracle is
 * the reference): the outer radial EM box scheme (Eqs. em_r_open_bx/bt), the
 * outer radial axion ghost, the exact space/time centring of the axion
 * current j_a (Sec. 2.2, Eqs. jax/jar/jat) beyond its energy-exchange
 * identity, and the zero-gradient extrapolation of S_a / j_a neighbours
 * beyond the last row.
 */
#define _USE_MATH_DEFINES
#include <complex.h>
#ifdef _OPENMP
#include <omp.h>
#endif
#include <math.h>
#include <stdlib.h>
#include <string.h>

#ifdef ORA_EXTENDED
/* Extended-precision build (liboracle_ext.so): the same arithmetic with
 * long double, used as the reference for FP64 parity where the paper's
 * form of E.B subtracts nearly equal products. */
typedef long double complex cplx;
#define RE(z) creall(z)
#define IM(z) cimagl(z)
#define CONJ(z) conjl(z)
#else
typedef double complex cplx;
#define RE(z) creal(z)
#define IM(z) cimag(z)
#define CONJ(z) conj(z)
#endif

enum {
  ORA_AXION = 1,          /* advance phi, T_a (Sec. 2.2)                     */
  ORA_AREM = 2,           /* advance the axion-regenerated fields (Sec. 2.2) */
  ORA_MOVING_WINDOW = 4,  /* window moves one cell per step                   */
  ORA_X_PERIODIC = 8,     /* periodic x (test mode for dispersion pins)       */
  ORA_R_CLOSED = 16,      /* conducting wall / Neumann axion at r = nr dr     */
  ORA_AXION_R_PRINTED = 1024  /* test reading: the outer phi row by the paper's
                                 three-level update as printed (see below)    */
};

enum { F_TRP, F_TRM, F_TTP, F_TTM, F_EX, F_BX, F_PHI, F_TAP, F_TAM,
       F_TRP1, F_TRM1, F_TTP1, F_TTM1, F_EX1, F_BX1, N_FIELDS };

typedef struct {
  int nx, nr, M;
  double h, dr, m_a, g;
  int flags;
  size_t plane; /* M*nx*nr */
  /* laser injection at x_min (NULL: none): the inflow characteristics
   * T_r^+ and T_th^- of the exterior cell -1 at time n, [M][nr] each */
  const cplx *in_rp, *in_tm;
} P;

static inline size_t ix(const P *p, int m, int i, int j) {
  return ((size_t)m * p->nx + (size_t)i) * p->nr + (size_t)j;
}
static inline int periodic(const P *p) { return (p->flags & ORA_X_PERIODIC) != 0; }

/* Value of a cell-located field; cells outside the box read as zero (open
 * boundary, Eq. em_x_open) or wrap (periodic test mode). */
static inline cplx cellv(const P *p, const cplx *a, int m, int i, int j) {
  if (periodic(p)) i = (i % p->nx + p->nx) % p->nx;
  else if (i < 0 || i >= p->nx) return 0;
  return a[ix(p, m, i, j)];
}
/* The exterior cell -1 behind x_min as seen by the shift into cell 0: the
 * open boundary of Eq. em_x_open has T_r^+ = T_th^- = 0 there; with laser
 * injection those two inflow characteristics take the prescribed values
 * (the outgoing T_r^-, T_th^+ stay zero outside). */
static inline cplx cell_in(const P *p, const cplx *a, const cplx *inflow, int m, int i, int j) {
  if (!periodic(p) && i == -1 && inflow) return inflow[(size_t)m * p->nr + j];
  return cellv(p, a, m, i, j);
}
static inline int real_face(const P *p, int f) {
  if (periodic(p)) return 1;
  return f >= 0 && f <= p->nx - 2;
}
/* Value of a face-located field; non-existent faces read as zero. */
static inline cplx facev(const P *p, const cplx *a, int m, int f, int j) {
  if (periodic(p)) f = (f % p->nx + p->nx) % p->nx;
  else if (f < 0 || f > p->nx - 2) return 0;
  if (!a) return 0;
  return a[ix(p, m, f, j)];
}
static inline double r_int(const P *p, int j) { return j * p->dr; }
static inline double r_half(const P *p, int j) { return (j + 0.5) * p->dr; }

/* ------------------------------------------------------------------------
 * Mode convolution C_m{A, B} (Sec. 2.2, Eq. mode_convolution).  A and B are
 * given per retained mode k = 0..M-1; negative modes are complex conjugates
 * (Eq. fourier_decomp).  k = 0 and l = 0 take part in all three sums.
 * ---------------------------------------------------------------------- */
static cplx mode_conv(int M, int m, const cplx *A, const cplx *B) {
  if (m == 0) {
    cplx s = A[0] * B[0];
    for (int k = 1; k < M; k++) s += 0.5 * RE(A[k] * CONJ(B[k]));
    return s;
  }
  cplx s = 0;
  for (int k = 0; k < M; k++)          /* k + l = m */
    for (int l = 0; l < M; l++)
      if (k + l == m) s += A[k] * B[l];
  for (int k = 0; k < M; k++)          /* k - l = m : A^(k) B^(-l) */
    for (int l = 0; l < M; l++)
      if (k - l == m) s += A[k] * CONJ(B[l]);
  for (int k = 0; k < M; k++)          /* l - k = m : A^(-k) B^(l) */
    for (int l = 0; l < M; l++)
      if (l - k == m) s += CONJ(A[k]) * B[l];
  return 0.5 * s;
}

/* exported for the quadrature pin */
/* Threads of the OpenMP loops (for timing the oracle on 1 thread and on all
 * cores); n <= 0 leaves the runtime's default.  Returns the count in force. */
int ora_set_threads(int n) {
#ifdef _OPENMP
  if (n > 0) omp_set_num_threads(n);
  return omp_get_max_threads();
#else
  (void)n;
  return 1;
#endif
}

void ora_mode_conv(int M, const double *A, const double *B, double *out) {
  cplx a[8], b[8];
  for (int k = 0; k < M && k < 8; k++) {
    a[k] = A[2 * k] + I * A[2 * k + 1];
    b[k] = B[2 * k] + I * B[2 * k + 1];
  }
  for (int m = 0; m < M; m++) {
    cplx r = mode_conv(M, m, a, b);
    out[2 * m] = (double)RE(r);
    out[2 * m + 1] = (double)IM(r);
  }
}

/* ------------------------------------------------------------------------
 * Mode products of many retained modes at many points (Sec. 3.3): for each
 * point q, out^(m) = sum_p w_p C_m{A_p, B_p}, m = 0..M-1.  A, B: [npairs][M]
 * [npts] complex, out: [M][npts].
 *   ora_mode_products: the convolution sums of Eq. mode_convolution;
 *   ora_mode_products_theta: the theta-grid procedure of Sec. 3.3 with
 *   ntheta equally spaced angles theta_s = 2 pi s / ntheta: each field
 *   F(theta_s) = Re sum_k F^(k) e^{-i k theta_s} (Eq. fourier_decomp), the
 *   products summed over the pairs pointwise, projected back by
 *   C_m = (2 / ntheta) sum_s P(theta_s) e^{i m theta_s}, halved for m = 0.
 *   Plain DFT sums (no FFT): the reference for the transform-based kernels.
 * ---------------------------------------------------------------------- */
static cplx load_c(const double *a, size_t q) { return a[2 * q] + I * a[2 * q + 1]; }

int ora_mode_products(int M, int npairs, int npts, const double *A, const double *B, const double *w,
                      double *out) {
  if (M < 1 || npairs < 1 || npts < 0) return -1;
  cplx *a = malloc(sizeof(cplx) * M), *b = malloc(sizeof(cplx) * M);
  if (!a || !b) { free(a); free(b); return -2; }
  for (int q = 0; q < npts; q++)
    for (int m = 0; m < M; m++) {
      cplx s = 0;
      for (int p = 0; p < npairs; p++) {
        for (int k = 0; k < M; k++) {
          a[k] = load_c(A, ((size_t)p * M + k) * npts + q);
          b[k] = load_c(B, ((size_t)p * M + k) * npts + q);
        }
        s += w[p] * mode_conv(M, m, a, b);
      }
      out[2 * ((size_t)m * npts + q)] = (double)RE(s);
      out[2 * ((size_t)m * npts + q) + 1] = (double)IM(s);
    }
  free(a); free(b);
  return 0;
}

int ora_mode_products_theta(int M, int npairs, int npts, int ntheta, const double *A, const double *B,
                            const double *w, double *out) {
  if (M < 1 || npairs < 1 || npts < 0 || ntheta < 1) return -1;
  for (int q = 0; q < npts; q++) {
    for (int m = 0; m < M; m++) {
      cplx c = 0;
      for (int s_ = 0; s_ < ntheta; s_++) {
        const double th = 2.0 * 3.14159265358979323846 * s_ / ntheta;
        double P = 0;
        for (int p = 0; p < npairs; p++) {
          double fa = 0, fb = 0;
          for (int k = 0; k < M; k++) {
            const cplx ak = load_c(A, ((size_t)p * M + k) * npts + q);
            const cplx bk = load_c(B, ((size_t)p * M + k) * npts + q);
            fa += (double)RE(ak * cexp(-I * (double)k * th));
            fb += (double)RE(bk * cexp(-I * (double)k * th));
          }
          P += w[p] * fa * fb;
        }
        c += P * cexp(I * (double)m * th);
      }
      c *= 2.0 / ntheta;
      if (m == 0) c *= 0.5;
      out[2 * ((size_t)m * npts + q)] = (double)RE(c);
      out[2 * ((size_t)m * npts + q) + 1] = (double)IM(c);
    }
  }
  return 0;
}

/* ------------------------------------------------------------------------
 * Transverse field reconstruction (Eq. reconstruct_fields):
 *   E_r = (T_r^+ + T_r^-)/2, B_th = (T_r^+ - T_r^-)/2c,
 *   E_th = (T_th^+ + T_th^-)/2, B_r = (T_th^+ - T_th^-)/2c.
 * ---------------------------------------------------------------------- */
typedef struct { cplx *Er, *Bt, *Et, *Br; } Transverse;

static void reconstruct(const P *p, const cplx *Trp, const cplx *Trm,
                        const cplx *Ttp, const cplx *Ttm, Transverse *t) {
  for (size_t q = 0; q < p->plane; q++) {
    t->Er[q] = 0.5 * (Trp[q] + Trm[q]);
    t->Bt[q] = 0.5 * (Trp[q] - Trm[q]);
    t->Et[q] = 0.5 * (Ttp[q] + Ttm[q]);
    t->Br[q] = 0.5 * (Ttp[q] - Ttm[q]);
  }
}

/* ------------------------------------------------------------------------
 * One QDS EM step (Sec. 2.1) on one field group.  Currents are given at the
 * faces where the update needs them: jx at (i+1/2, j, n), jr at
 * (i+1/2, j+1/2, n+1/2), jt at (i+1/2, j, n+1/2).  NULL means zero.
 * Order: longitudinal leapfrog E_x, B_x to n+1/2 from the transverse fields
 * at n (Eq. Ex_update), then the characteristic shift of T to n+1 with
 * sources at n+1/2 (Eqs. Trp/Trm/Ttp/Ttm_update).
 * ---------------------------------------------------------------------- */
static void em_step(const P *p, const cplx *Trp, const cplx *Trm,
                    const cplx *Ttp, const cplx *Ttm, const cplx *Ex,
                    const cplx *Bx, const cplx *jx, const cplx *jr,
                    const cplx *jt, cplx *nTrp, cplx *nTrm, cplx *nTtp,
                    cplx *nTtm, cplx *nEx, cplx *nBx, const Transverse *t) {
  const int nx = p->nx, nr = p->nr, M = p->M;
  const double h = p->h, dr = p->dr;
  const int closed = (p->flags & ORA_R_CLOSED) != 0;
  const int J = nr - 1; /* last integer row; last half row is J + 1/2 */

  /* --- E_x and B_x leapfrog (Eqs. Ex_update, Gammax_explicit,
   *     Phix_explicit, axis_Ex). --------------------------------------- */
#pragma omp parallel for collapse(2) schedule(static)
  for (int m = 0; m < M; m++)
    for (int f = 0; f < nx; f++) {
      if (!real_face(p, f)) {
        for (int j = 0; j < nr; j++) nEx[ix(p, m, f, j)] = nBx[ix(p, m, f, j)] = 0;
        continue;
      }
      const int c0 = f, c1 = f + 1; /* the two cells around face f */
      for (int j = 0; j < nr; j++) {
        /* E_x at (i+1/2, j) */
        cplx Gx;
        if (j == 0) {
          if (m == 0) {
            /* Eq. axis_Ex: dE_x/dt = 2 c^2 dB_th/dr - j_x, dB_th/dr ~ 2 B_th(1/2)/dr,
             * B_th(i+1/2, 1/2) from the two neighbouring cells. */
            cplx Bth = 0.5 * (cellv(p, t->Bt, m, c0, 0) + cellv(p, t->Bt, m, c1, 0));
            Gx = 2.0 * (2.0 / dr) * Bth - facev(p, jx, m, f, 0);
            nEx[ix(p, m, f, 0)] = Ex[ix(p, m, f, 0)] + h * Gx;
          } else {
            nEx[ix(p, m, f, 0)] = 0; /* F_x^(m!=0)(r=0) = 0 (Sec. 2.3) */
          }
        } else {
          /* (1/r) d(r B_th)/dr = B_th/r + dB_th/dr, with B_th averaged onto
           * (i+1/2, j) by the four-point stencil and dB_th/dr by the centred
           * difference of the same samples (Sec. 2.1). */
          cplx b_lo = cellv(p, t->Bt, m, c0, j - 1) + cellv(p, t->Bt, m, c1, j - 1);
          cplx b_hi = cellv(p, t->Bt, m, c0, j) + cellv(p, t->Bt, m, c1, j);
          cplx Bth_avg = 0.25 * (b_lo + b_hi);
          cplx dBth = (b_hi - b_lo) / (2.0 * dr);
          cplx Br_avg = 0.5 * (cellv(p, t->Br, m, c0, j) + cellv(p, t->Br, m, c1, j));
          double rj = r_int(p, j);
          Gx = Bth_avg / rj + dBth + I * (double)m * Br_avg / rj - facev(p, jx, m, f, j);
          nEx[ix(p, m, f, j)] = Ex[ix(p, m, f, j)] + h * Gx;
        }
        /* B_x at (i+1/2, j+1/2) */
        if (j < J || closed) {
          cplx e_lo = cellv(p, t->Et, m, c0, j) + cellv(p, t->Et, m, c1, j);
          cplx e_hi = (j < J) ? cellv(p, t->Et, m, c0, j + 1) + cellv(p, t->Et, m, c1, j + 1)
                              : 0; /* conducting wall: E_th = 0 at r = nr dr */
          cplx Eth_avg = 0.25 * (e_lo + e_hi);
          cplx dEth = (e_hi - e_lo) / (2.0 * dr);
          cplx Er_avg = 0.5 * (cellv(p, t->Er, m, c0, j) + cellv(p, t->Er, m, c1, j));
          double rh = r_half(p, j);
          cplx Px = -(Eth_avg / rh + dEth) - I * (double)m * Er_avg / rh;
          nBx[ix(p, m, f, j)] = Bx[ix(p, m, f, j)] + h * Px;
        }
      }
    }

  if (!closed) {
    /* Outer half row J+1/2: Eq. em_r_open_bx,
     *   (d_t + c d_r) B_x = (c/2) d_x B_r - (E_th + i m E_r)/(2r) - j_th/(2c),
     * by the box scheme on [r_{J-1/2}, r_{J+1/2}] x [t^{n-1/2}, t^{n+1/2}],
     * centred at (i+1/2, r_J, t^n), right-hand side from time-n fields. */
#pragma omp parallel for collapse(2) schedule(static)
    for (int m = 0; m < M; m++)
      for (int f = 0; f < nx; f++) {
        if (!real_face(p, f)) continue;
        const int c0 = f, c1 = f + 1;
        double rJ = r_int(p, J);
        cplx dxBr = (cellv(p, t->Br, m, c1, J) - cellv(p, t->Br, m, c0, J)) / h;
        cplx Eth = 0.5 * (cellv(p, t->Et, m, c0, J) + cellv(p, t->Et, m, c1, J));
        cplx Er = 0.25 * (cellv(p, t->Er, m, c0, J - 1) + cellv(p, t->Er, m, c0, J) +
                          cellv(p, t->Er, m, c1, J - 1) + cellv(p, t->Er, m, c1, J));
        cplx R = 0.5 * dxBr - (Eth + I * (double)m * Er) / (2.0 * rJ) - 0.5 * facev(p, jt, m, f, J);
        cplx bi_new = nBx[ix(p, m, f, J - 1)];
        cplx bo_old = Bx[ix(p, m, f, J)], bi_old = Bx[ix(p, m, f, J - 1)];
        double a = 1.0 / (2.0 * h), b = 1.0 / (2.0 * dr);
        nBx[ix(p, m, f, J)] =
            (R - bi_new * (a - b) + (bo_old + bi_old) * a - (bo_old - bi_old) * b) / (a + b);
      }
  }

  /* --- Characteristic shift of the transport variables (Eqs. Trp_update,
   *     Trm_update, Ttp_update, Ttm_update) with the face sources
   *     Gamma_r +- c Phi_r at (i+1/2, j+1/2) and Gamma_th +- c Phi_th at
   *     (i+1/2, j), using E_x, B_x at n+1/2. ------------------------------ */
#pragma omp parallel for collapse(2) schedule(static)
  for (int m = 0; m < M; m++)
    for (int c = 0; c < nx; c++) {
      for (int j = 0; j < nr; j++) {
        /* T_r^{+-} at half row j */
        if (j < J || closed) {
          for (int s = 0; s < 2; s++) { /* s=0: T_r^+ from face c-1; s=1: T_r^- from face c */
            int f = (s == 0) ? c - 1 : c;
            cplx src = 0;
            if (real_face(p, f)) {
              double rh = r_half(p, j);
              cplx Gr = -I * (double)m * facev(p, nBx, m, f, j) / rh - facev(p, jr, m, f, j);
              cplx ex_hi = (j < J) ? facev(p, nEx, m, f, j + 1) : 0; /* wall: E_x = 0 */
              cplx Pr = (ex_hi - facev(p, nEx, m, f, j)) / dr;
              src = (s == 0) ? Gr + Pr : Gr - Pr;
            }
            if (s == 0) nTrp[ix(p, m, c, j)] = cell_in(p, Trp, p->in_rp, m, c - 1, j) + h * src;
            else nTrm[ix(p, m, c, j)] = cellv(p, Trm, m, c + 1, j) + h * src;
          }
        }
        /* T_th^{+-} at integer row j */
        if (j == 0 && m != 1) { /* F_r = F_th = 0 on axis for m != 1 (Sec. 2.3) */
          nTtp[ix(p, m, c, 0)] = 0;
          nTtm[ix(p, m, c, 0)] = 0;
          continue;
        }
        for (int s = 0; s < 2; s++) { /* s=0: T_th^+ from face c; s=1: T_th^- from face c-1 */
          int f = (s == 0) ? c : c - 1;
          cplx src = 0;
          if (real_face(p, f)) {
            cplx Gt, Pt;
            if (j == 0) {
              /* Eq. axis_Ttheta (m = 1): dB_x/dr ~ 2 B_x(1/2)/dr,
               * dE_x/dr ~ (E_x(1) - E_x(0))/dr, and i m E_x / r -> i dE_x/dr. */
              Gt = -(2.0 / dr) * facev(p, nBx, m, f, 0) - facev(p, jt, m, f, 0);
              Pt = I * (facev(p, nEx, m, f, 1) - facev(p, nEx, m, f, 0)) / dr;
            } else {
              Gt = -(facev(p, nBx, m, f, j) - facev(p, nBx, m, f, j - 1)) / dr - facev(p, jt, m, f, j);
              Pt = I * (double)m * facev(p, nEx, m, f, j) / r_int(p, j);
            }
            src = (s == 0) ? Gt + Pt : Gt - Pt;
          }
          if (s == 0) nTtp[ix(p, m, c, j)] = cellv(p, Ttp, m, c + 1, j) + h * src;
          else nTtm[ix(p, m, c, j)] = cell_in(p, Ttm, p->in_tm, m, c - 1, j) + h * src;
        }
      }
    }

  if (!closed) {
    /* Outer half row J+1/2 (Sec. 3.2, Eq. em_r_open_bt).  E_r = (T_r^+ + T_r^-)/2
     * is advanced by the characteristic shift with the Gamma_r source only
     * (Phi_r = dE_x/dr would need E_x beyond the last row; it enters E_r only
     * at second order).  B_th is advanced by the box scheme of
     *   (d_t + c d_r) B_th = -(1/2) d_x E_r - (c/2r)(B_th + i m B_r) + j_x/(2c)
     * on [r_{J-1/2}, r_{J+1/2}] x [t^n, t^{n+1}], right-hand side from time-n
     * fields.  Then T_r^{+-} = E_r +- c B_th. */
#pragma omp parallel for collapse(2) schedule(static)
    for (int m = 0; m < M; m++)
      for (int c = 0; c < nx; c++) {
        double rh = r_half(p, J), rJ = r_int(p, J);
        cplx Gr_l = 0, Gr_r = 0;
        if (real_face(p, c - 1))
          Gr_l = -I * (double)m * facev(p, nBx, m, c - 1, J) / rh - facev(p, jr, m, c - 1, J);
        if (real_face(p, c))
          Gr_r = -I * (double)m * facev(p, nBx, m, c, J) / rh - facev(p, jr, m, c, J);
        cplx Tp = cell_in(p, Trp, p->in_rp, m, c - 1, J) + h * Gr_l;
        cplx Tm = cellv(p, Trm, m, c + 1, J) + h * Gr_r;
        cplx Er_new = 0.5 * (Tp + Tm);

        cplx Er_l = 0.5 * (cellv(p, t->Er, m, c - 1, J - 1) + cellv(p, t->Er, m, c - 1, J));
        if (c == 0 && !periodic(p) && p->in_rp) /* E_r = (T_r^+ + T_r^-)/2 of the exterior cell */
          Er_l = 0.25 * (p->in_rp[(size_t)m * nr + J - 1] + p->in_rp[(size_t)m * nr + J]);
        cplx Er_r = 0.5 * (cellv(p, t->Er, m, c + 1, J - 1) + cellv(p, t->Er, m, c + 1, J));
        cplx dxEr = (Er_r - Er_l) / (2.0 * h);
        cplx Bth = 0.5 * (cellv(p, t->Bt, m, c, J - 1) + cellv(p, t->Bt, m, c, J));
        cplx Br = cellv(p, t->Br, m, c, J);
        cplx jxc = 0.5 * (facev(p, jx, m, c - 1, J) + facev(p, jx, m, c, J));
        cplx R = -0.5 * dxEr - (Bth + I * (double)m * Br) / (2.0 * rJ) + 0.5 * jxc;
        cplx bi_new = 0.5 * (nTrp[ix(p, m, c, J - 1)] - nTrm[ix(p, m, c, J - 1)]);
        cplx bo_old = t->Bt[ix(p, m, c, J)], bi_old = t->Bt[ix(p, m, c, J - 1)];
        double a = 1.0 / (2.0 * h), b = 1.0 / (2.0 * dr);
        cplx Bt_new =
            (R - bi_new * (a - b) + (bo_old + bi_old) * a - (bo_old - bi_old) * b) / (a + b);
        nTrp[ix(p, m, c, J)] = Er_new + Bt_new;
        nTrm[ix(p, m, c, J)] = Er_new - Bt_new;
      }
  }
}

/* ------------------------------------------------------------------------
 * The full step.
 * ---------------------------------------------------------------------- */
static cplx *fld(cplx *base, const P *p, int f) { return base + (size_t)f * p->plane; }
static cplx *to_cplx(const double *d, size_t n);

/* Value beyond the last row used by averages that reach one row past it:
 * zero-gradient for the open boundary, zero for the conducting wall. */
static inline cplx row_or_edge(const P *p, const cplx *a, int m, int c, int j, int face) {
  if (j >= p->nr) {
    if (p->flags & ORA_R_CLOSED) return 0;
    j = p->nr - 1;
  }
  return face ? facev(p, a, m, c, j) : cellv(p, a, m, c, j);
}

/* Mirror across the axis of a scalar sampled on half rows (phi and its
 * derivatives): value at row -1/2 equals (-1)^m times the value at +1/2
 * (the parity reading of Sec. 2.3, consistent with Eq. axis_Ttheta). */
static inline double parity(int m) { return (m & 1) ? -1.0 : 1.0; }

static int step_once(const P *p, cplx *S, const cplx *jx, const cplx *jrc, const cplx *jtc,
                     const cplx *sext) {
  const int nx = p->nx, nr = p->nr, M = p->M;
  const double h = p->h, dr = p->dr, m_a = p->m_a, g = p->g;
  const int flags = p->flags;
  const size_t pl = p->plane;
  cplx *phiprev = S + (size_t)N_FIELDS * pl; /* [M][nx]: phi at the outer row, time n-1 */
  const int J = nr - 1;
  const int closed = (flags & ORA_R_CLOSED) != 0;

  cplx *N = calloc((size_t)N_FIELDS * pl + (size_t)M * nx, sizeof(cplx));
  cplx *tmp = calloc(12 * pl, sizeof(cplx));
  if (!N || !tmp) { free(N); free(tmp); return -2; }
  Transverse t0 = {tmp, tmp + pl, tmp + 2 * pl, tmp + 3 * pl};
  Transverse t0n = {tmp + 4 * pl, tmp + 5 * pl, tmp + 6 * pl, tmp + 7 * pl};
  cplx *jrf = tmp + 8 * pl, *jtf = tmp + 9 * pl, *Sa = tmp + 10 * pl, *Ga = tmp + 11 * pl;

  /* ---- EM0: currents x-averaged onto the faces where the T update needs
   *      them (Sec. 3.1, last paragraph). ------------------------------ */
  for (int m = 0; m < M; m++)
    for (int f = 0; f < nx; f++)
      for (int j = 0; j < nr; j++) {
        size_t q = ix(p, m, f, j);
        jrf[q] = jtf[q] = 0;
        if (!real_face(p, f)) continue;
        if (jrc) jrf[q] = 0.5 * (cellv(p, jrc, m, f, j) + cellv(p, jrc, m, f + 1, j));
        if (jtc) jtf[q] = 0.5 * (cellv(p, jtc, m, f, j) + cellv(p, jtc, m, f + 1, j));
      }
  reconstruct(p, fld(S, p, F_TRP), fld(S, p, F_TRM), fld(S, p, F_TTP), fld(S, p, F_TTM), &t0);
  em_step(p, fld(S, p, F_TRP), fld(S, p, F_TRM), fld(S, p, F_TTP), fld(S, p, F_TTM),
          fld(S, p, F_EX), fld(S, p, F_BX), jx, jrf, jtf,
          fld(N, p, F_TRP), fld(N, p, F_TRM), fld(N, p, F_TTP), fld(N, p, F_TTM),
          fld(N, p, F_EX), fld(N, p, F_BX), &t0);
  reconstruct(p, fld(N, p, F_TRP), fld(N, p, F_TRM), fld(N, p, F_TTP), fld(N, p, F_TTM), &t0n);

  const cplx *Ex = fld(S, p, F_EX), *Bx = fld(S, p, F_BX);
  const cplx *nEx = fld(N, p, F_EX), *nBx = fld(N, p, F_BX);
  const cplx *phi = fld(S, p, F_PHI), *Tap = fld(S, p, F_TAP), *Tam = fld(S, p, F_TAM);
  cplx *nphi = fld(N, p, F_PHI), *nTap = fld(N, p, F_TAP), *nTam = fld(N, p, F_TAM);
  cplx *nphiprev = N + (size_t)N_FIELDS * pl;

  if (flags & (ORA_AXION | ORA_AREM)) {
    /* ---- Axion source S_a^(m) = sum_alpha C_m{E_alpha, B_alpha} at
     *      (i+1/2, j+1/2, n) (Eqs. source_mode_zero/_m); every component is
     *      first averaged onto that point, E_x and B_x also in time. ------ */
#pragma omp parallel for collapse(2) schedule(static)
    for (int f = 0; f < nx; f++)
      for (int j = 0; j < nr; j++) {
        cplx eX[8], bX[8], eR[8], bR[8], eT[8], bT[8];
        for (int k = 0; k < M; k++) {
          eX[k] = 0.25 * (facev(p, Ex, k, f, j) + row_or_edge(p, Ex, k, f, j + 1, 1) +
                          facev(p, nEx, k, f, j) + row_or_edge(p, nEx, k, f, j + 1, 1));
          bX[k] = 0.5 * (facev(p, Bx, k, f, j) + facev(p, nBx, k, f, j));
          eR[k] = 0.5 * (cellv(p, t0.Er, k, f, j) + cellv(p, t0.Er, k, f + 1, j));
          bT[k] = 0.5 * (cellv(p, t0.Bt, k, f, j) + cellv(p, t0.Bt, k, f + 1, j));
          eT[k] = 0.25 * (cellv(p, t0.Et, k, f, j) + cellv(p, t0.Et, k, f + 1, j) +
                          row_or_edge(p, t0.Et, k, f, j + 1, 0) + row_or_edge(p, t0.Et, k, f + 1, j + 1, 0));
          bR[k] = 0.25 * (cellv(p, t0.Br, k, f, j) + cellv(p, t0.Br, k, f + 1, j) +
                          row_or_edge(p, t0.Br, k, f, j + 1, 0) + row_or_edge(p, t0.Br, k, f + 1, j + 1, 0));
        }
        for (int m = 0; m < M; m++) {
          cplx s = 0;
          if (real_face(p, f)) {
            s = mode_conv(M, m, eX, bX) + mode_conv(M, m, eR, bR) + mode_conv(M, m, eT, bT);
            if (sext) s += sext[ix(p, m, f, j)];
          }
          Sa[ix(p, m, f, j)] = s;
        }
      }

    /* ---- Exterior ghost of phi beyond the outermost half row N from the
     *      outgoing condition (d_t + c d_r) phi = 0 (Eq. axion_r_sommerfeld),
     *      centred at r_N as in Eq. axion_r_ghost, with d_t phi taken half a
     *      step back, (phi_N^n - phi_N^{n-1})/dt, so the ghost is explicit:
     *        phi_{N+1} = phi_{N-1} - (2 dr / c dt)(phi_N^n - phi_N^{n-1}).
     *      The paper's explicit three-level row update (Eq. axion_r_update)
     *      is not used: with c dt = dx its x-Laplacian sits at Courant number
     *      one and, with any radial term added, the x-Nyquist mode grows
     *      (|lambda| ~ 1.16 at dr = 5 dx).  The outer row is advanced by the
     *      same transport as the interior. */
    cplx *ghost = calloc((size_t)M * nx, sizeof(cplx));
    for (int m = 0; m < M; m++)
      for (int f = 0; f < nx; f++) {
        size_t q = (size_t)m * nx + f;
        if (!real_face(p, f) || closed) continue;
        ghost[q] = phi[ix(p, m, f, J - 1)] - (2.0 * dr / h) * (phi[ix(p, m, f, J)] - phiprev[q]);
      }

    /* ---- Gamma_a at (i+1/2, j+1/2, n) (Sec. 2.2): centred radial
     *      Laplacian, mass term and g S_a. --------------------------------- */
    for (int m = 0; m < M; m++)
      for (int f = 0; f < nx; f++)
        for (int j = 0; j < nr; j++) {
          size_t q = ix(p, m, f, j);
          if (!real_face(p, f)) { Ga[q] = 0; continue; }
          cplx pc = phi[q];
          cplx pm = (j == 0) ? parity(m) * phi[ix(p, m, f, 0)] : phi[ix(p, m, f, j - 1)];
          cplx pp_;
          if (j < J) pp_ = phi[ix(p, m, f, j + 1)];
          else pp_ = closed ? pc : ghost[(size_t)m * nx + f];
          double rh = r_half(p, j);
          cplx d2 = (pp_ - 2.0 * pc + pm) / (dr * dr);
          cplx d1 = (pp_ - pm) / (2.0 * dr);
          Ga[q] = d2 + d1 / rh - (double)(m * m) / (rh * rh) * pc - m_a * m_a * pc + g * Sa[q];
        }

    /* ---- T_a shift (Eqs. Ta_plus_update, Ta_minus_update) and phi update
     *      (Eq. phi_update). -------------------------------------------- */
    for (int m = 0; m < M; m++)
      for (int c = 0; c < nx; c++)
        for (int j = 0; j < nr; j++) {
          nTap[ix(p, m, c, j)] = cellv(p, Tap, m, c - 1, j) + h * facev(p, Ga, m, c - 1, j);
          nTam[ix(p, m, c, j)] = cellv(p, Tam, m, c + 1, j) + h * facev(p, Ga, m, c, j);
        }
    for (int m = 0; m < M; m++)
      for (int f = 0; f < nx; f++) {
        for (int j = 0; j < nr; j++) {
          size_t q = ix(p, m, f, j);
          if (!real_face(p, f)) { nphi[q] = 0; continue; }
          nphi[q] = phi[q] + (h / 4.0) * (cellv(p, nTam, m, f + 1, j) + cellv(p, nTam, m, f, j) +
                                          cellv(p, nTap, m, f + 1, j) + cellv(p, nTap, m, f, j));
        }
        size_t q = (size_t)m * nx + f;
        nphiprev[q] = real_face(p, f) ? phi[ix(p, m, f, J)] : 0;
      }
    if ((flags & ORA_AXION_R_PRINTED) && !closed) {
      /* Test reading, used only to pin why the default reading above
       * departs from the paper: the outermost phi row by the explicit
       * three-level update exactly as printed (Eq. axion_r_update, Sec. 3.2),
       *   A phi^{n+1} = -(1/dt^2 - c/(dr dt) - c/(2 r_N dt)) phi^{n-1}
       *                 + (2/dt^2) phi^n + R^n,
       *   A = 1/dt^2 + c/(dr dt) + c/(2 r_N dt),
       *   R^n = c^2 (phi_{i+1} - 2 phi_i + phi_{i-1})/dx^2 - m^2 c^2 phi/r_N^2
       *         + (2 c^2/dr^2)(phi_{N-1} - phi_N) - m_a^2 phi + g S_a,
       * with r_N the radius of the outermost half row.  "The same update at
       * the auxiliary half time level" is read as T_a^{+-} of that row
       * following from phi: T_a^{+-} = d_t phi -+ d_x phi at (cell, n+1/2),
       * centred from the faces around the cell and the levels n, n+1. */
      const double rN = r_half(p, J);
      const double A = 1.0 / (h * h) + 1.0 / (dr * h) + 1.0 / (2.0 * rN * h);
      const double Bc = 1.0 / (h * h) - 1.0 / (dr * h) - 1.0 / (2.0 * rN * h);
      for (int m = 0; m < M; m++)
        for (int f = 0; f < nx; f++) {
          size_t q = ix(p, m, f, J);
          if (!real_face(p, f)) continue;
          cplx pc = phi[q];
          cplx lapx = (facev(p, phi, m, f + 1, J) - 2.0 * pc + facev(p, phi, m, f - 1, J)) / (h * h);
          cplx R = lapx - (double)(m * m) / (rN * rN) * pc + (2.0 / (dr * dr)) * (phi[ix(p, m, f, J - 1)] - pc) -
                   m_a * m_a * pc + g * Sa[q];
          nphi[q] = (-Bc * phiprev[(size_t)m * nx + f] + (2.0 / (h * h)) * pc + R) / A;
        }
      for (int m = 0; m < M; m++)
        for (int c = 0; c < nx; c++) {
          cplx dt = 0.5 * ((facev(p, nphi, m, c - 1, J) - facev(p, phi, m, c - 1, J)) +
                           (facev(p, nphi, m, c, J) - facev(p, phi, m, c, J))) / h;
          cplx dx = 0.5 * ((facev(p, nphi, m, c, J) - facev(p, nphi, m, c - 1, J)) +
                           (facev(p, phi, m, c, J) - facev(p, phi, m, c - 1, J))) / h;
          nTap[ix(p, m, c, J)] = dt - dx;
          nTam[ix(p, m, c, J)] = dt + dx;
        }
    }
    free(ghost);
  }

  if (flags & ORA_AREM) {
    /* ---- Axion current j_a = g (B0 d_t phi - E0 x grad phi) (Eqs. jax_mode,
     *      jar_mode, jat_mode) at the points the AREM update needs:
     *      j_a,x at (i+1/2, j, n); j_a,r at (i+1/2, j+1/2, n+1/2);
     *      j_a,th at (i+1/2, j, n+1/2).  (d_th phi)^(l) = -i l phi^(l). ---- */
    cplx *jax = calloc(3 * pl, sizeof(cplx));
    cplx *jar = jax + pl, *jat = jax + 2 * pl;
#pragma omp parallel for collapse(2) schedule(static)
    for (int f = 0; f < nx; f++)
      for (int j = 0; j < nr; j++) {
        if (!real_face(p, f)) continue;
        cplx bx[8], dtp[8], er[8], dth[8], et[8], drp[8];
        cplx br2[8], dtp2[8], et2[8], dxp2[8], ex2[8], dth2[8];
        cplx bt3[8], dtp3[8], ex3[8], drp3[8], er3[8], dxp3[8];
        for (int k = 0; k < M; k++) {
          double par = parity(k);
          /* d_t phi at a half row, time n: (c/2)(T_a^+ + T_a^-) (Eq. phi_update)
           * averaged over the two cells around face f and the levels n -+ 1/2. */
#define DTPHI_N(jj) (0.125 * (cellv(p, Tap, k, f, jj) + cellv(p, Tam, k, f, jj) +        \
                              cellv(p, Tap, k, f + 1, jj) + cellv(p, Tam, k, f + 1, jj) + \
                              cellv(p, nTap, k, f, jj) + cellv(p, nTam, k, f, jj) +      \
                              cellv(p, nTap, k, f + 1, jj) + cellv(p, nTam, k, f + 1, jj)))
          /* ---- j_a,x at (i+1/2, j, n) ---- */
          {
            cplx bx_lo = (j == 0) ? par * 0.5 * (Bx[ix(p, k, f, 0)] + nBx[ix(p, k, f, 0)])
                                  : 0.5 * (Bx[ix(p, k, f, j - 1)] + nBx[ix(p, k, f, j - 1)]);
            cplx bx_hi = 0.5 * (Bx[ix(p, k, f, j)] + nBx[ix(p, k, f, j)]);
            bx[k] = 0.5 * (bx_lo + bx_hi);
            cplx dt_hi = DTPHI_N(j);
            cplx dt_lo = (j == 0) ? par * DTPHI_N(0) : DTPHI_N(j - 1);
            dtp[k] = 0.5 * (dt_lo + dt_hi);
            /* E_r on the half rows around row j, with the axis ghost at j = 0
             * from T_r^{+-}(-1/2) = 2i T_th^{-+}(0) - T_r^{+-}(1/2) (m = 1) and
             * -T_r(1/2) otherwise (Sec. 2.3). */
            cplx er_hi = 0.5 * (cellv(p, t0.Er, k, f, j) + cellv(p, t0.Er, k, f + 1, j));
            cplx er_lo;
            if (j > 0) er_lo = 0.5 * (cellv(p, t0.Er, k, f, j - 1) + cellv(p, t0.Er, k, f + 1, j - 1));
            else if (k == 1) er_lo = 0.5 * (2.0 * I * cellv(p, t0.Et, k, f, 0) - cellv(p, t0.Er, k, f, 0) +
                                            2.0 * I * cellv(p, t0.Et, k, f + 1, 0) - cellv(p, t0.Er, k, f + 1, 0));
            else er_lo = -er_hi;
            er[k] = 0.5 * (er_lo + er_hi);
            et[k] = 0.5 * (cellv(p, t0.Et, k, f, j) + cellv(p, t0.Et, k, f + 1, j));
            cplx ph_hi = phi[ix(p, k, f, j)];
            cplx ph_lo = (j == 0) ? par * phi[ix(p, k, f, 0)] : phi[ix(p, k, f, j - 1)];
            drp[k] = (ph_hi - ph_lo) / dr;
            /* (1/r) d_th phi at row j; on the axis its r -> 0 limit, which is
             * -i d_r phi^(1) for l = 1 and zero otherwise. */
            if (j > 0) dth[k] = -I * (double)k * 0.5 * (ph_lo + ph_hi) / r_int(p, j);
            else dth[k] = (k == 1) ? -I * (ph_hi - ph_lo) / dr : 0;
          }
          /* time-n+1/2 transverse fields: mean of levels n and n+1 */
#define ER5(c, jj) (0.5 * (cellv(p, t0.Er, k, c, jj) + cellv(p, t0n.Er, k, c, jj)))
#define BT5(c, jj) (0.5 * (cellv(p, t0.Bt, k, c, jj) + cellv(p, t0n.Bt, k, c, jj)))
#define ET5(c, jj) (0.5 * (row_or_edge(p, t0.Et, k, c, jj, 0) + row_or_edge(p, t0n.Et, k, c, jj, 0)))
#define BR5(c, jj) (0.5 * (row_or_edge(p, t0.Br, k, c, jj, 0) + row_or_edge(p, t0n.Br, k, c, jj, 0)))
#define DXPHI(jj) (0.25 * (cellv(p, nTam, k, f, jj) - cellv(p, nTap, k, f, jj) + \
                           cellv(p, nTam, k, f + 1, jj) - cellv(p, nTap, k, f + 1, jj)))
          /* ---- j_a,r at (i+1/2, j+1/2, n+1/2) ---- */
          {
            br2[k] = 0.25 * (BR5(f, j) + BR5(f + 1, j) + BR5(f, j + 1) + BR5(f + 1, j + 1));
            et2[k] = 0.25 * (ET5(f, j) + ET5(f + 1, j) + ET5(f, j + 1) + ET5(f + 1, j + 1));
            dtp2[k] = (nphi[ix(p, k, f, j)] - phi[ix(p, k, f, j)]) / h;
            dxp2[k] = DXPHI(j);
            ex2[k] = 0.5 * (facev(p, nEx, k, f, j) + row_or_edge(p, nEx, k, f, j + 1, 1));
            dth2[k] = -I * (double)k * 0.5 * (phi[ix(p, k, f, j)] + nphi[ix(p, k, f, j)]) / r_half(p, j);
          }
          /* ---- j_a,th at (i+1/2, j, n+1/2) ---- */
          {
            cplx bt_hi = 0.5 * (BT5(f, j) + BT5(f + 1, j));
            cplx bt_lo, er_hi = 0.5 * (ER5(f, j) + ER5(f + 1, j)), er_lo;
            if (j > 0) {
              bt_lo = 0.5 * (BT5(f, j - 1) + BT5(f + 1, j - 1));
              er_lo = 0.5 * (ER5(f, j - 1) + ER5(f + 1, j - 1));
            } else if (k == 1) {
              /* B_th(-1/2) = -2i B_r(0) - B_th(1/2); E_r(-1/2) = 2i E_th(0) - E_r(1/2) */
              cplx br0 = 0.5 * (BR5(f, 0) + BR5(f + 1, 0));
              cplx et0 = 0.5 * (ET5(f, 0) + ET5(f + 1, 0));
              bt_lo = -2.0 * I * br0 - bt_hi;
              er_lo = 2.0 * I * et0 - er_hi;
            } else {
              bt_lo = -bt_hi;
              er_lo = -er_hi;
            }
            bt3[k] = 0.5 * (bt_lo + bt_hi);
            er3[k] = 0.5 * (er_lo + er_hi);
            cplx dt_hi = (nphi[ix(p, k, f, j)] - phi[ix(p, k, f, j)]) / h;
            cplx dt_lo = (j == 0) ? par * dt_hi : (nphi[ix(p, k, f, j - 1)] - phi[ix(p, k, f, j - 1)]) / h;
            dtp3[k] = 0.5 * (dt_lo + dt_hi);
            ex3[k] = facev(p, nEx, k, f, j);
            cplx pb_hi = 0.5 * (phi[ix(p, k, f, j)] + nphi[ix(p, k, f, j)]);
            cplx pb_lo = (j == 0) ? par * pb_hi
                                  : 0.5 * (phi[ix(p, k, f, j - 1)] + nphi[ix(p, k, f, j - 1)]);
            drp3[k] = (pb_hi - pb_lo) / dr;
            cplx dx_hi = DXPHI(j);
            cplx dx_lo = (j == 0) ? par * dx_hi : DXPHI(j - 1);
            dxp3[k] = 0.5 * (dx_lo + dx_hi);
          }
#undef DTPHI_N
#undef ER5
#undef BT5
#undef ET5
#undef BR5
#undef DXPHI
        }
        for (int m = 0; m < M; m++) {
          size_t q = ix(p, m, f, j);
          jax[q] = g * (mode_conv(M, m, bx, dtp) - mode_conv(M, m, er, dth) + mode_conv(M, m, et, drp));
          jar[q] = g * (mode_conv(M, m, br2, dtp2) - mode_conv(M, m, et2, dxp2) + mode_conv(M, m, ex2, dth2));
          jat[q] = g * (mode_conv(M, m, bt3, dtp3) - mode_conv(M, m, ex3, drp3) + mode_conv(M, m, er3, dxp3));
        }
      }

    /* ---- AREM: the duplicate QDS step on (E1, B1) driven by j_a. ---- */
    Transverse t1 = {tmp, tmp + pl, tmp + 2 * pl, tmp + 3 * pl}; /* reuse t0 storage */
    reconstruct(p, fld(S, p, F_TRP1), fld(S, p, F_TRM1), fld(S, p, F_TTP1), fld(S, p, F_TTM1), &t1);
    P p1 = *p; /* the laser is injected into the EM field only */
    p1.in_rp = p1.in_tm = NULL;
    em_step(&p1, fld(S, p, F_TRP1), fld(S, p, F_TRM1), fld(S, p, F_TTP1), fld(S, p, F_TTM1),
            fld(S, p, F_EX1), fld(S, p, F_BX1), jax, jar, jat,
            fld(N, p, F_TRP1), fld(N, p, F_TRM1), fld(N, p, F_TTP1), fld(N, p, F_TTM1),
            fld(N, p, F_EX1), fld(N, p, F_BX1), &t1);
    free(jax);
  } else {
    memcpy(fld(N, p, F_TRP1), fld(S, p, F_TRP1), 6 * pl * sizeof(cplx));
  }
  if (!(flags & (ORA_AXION | ORA_AREM))) {
    memcpy(fld(N, p, F_PHI), fld(S, p, F_PHI), 3 * pl * sizeof(cplx));
    memcpy(nphiprev, phiprev, (size_t)M * nx * sizeof(cplx));
  }

  /* ---- Moving window: the box advances one cell; every field drops its
   *      rear column and gains a zero column at the front. ------------- */
  if (flags & ORA_MOVING_WINDOW) {
    for (int fi = 0; fi < N_FIELDS; fi++) {
      cplx *a = fld(N, p, fi);
      for (int m = 0; m < M; m++) {
        memmove(&a[ix(p, m, 0, 0)], &a[ix(p, m, 1, 0)], (size_t)(nx - 1) * nr * sizeof(cplx));
        memset(&a[ix(p, m, nx - 1, 0)], 0, (size_t)nr * sizeof(cplx));
      }
    }
    for (int m = 0; m < M; m++) {
      memmove(&nphiprev[(size_t)m * nx], &nphiprev[(size_t)m * nx + 1], (size_t)(nx - 1) * sizeof(cplx));
      nphiprev[(size_t)m * nx + nx - 1] = 0;
    }
  }

  memcpy(S, N, ((size_t)N_FIELDS * pl + (size_t)M * nx) * sizeof(cplx));
  free(N);
  free(tmp);
  return 0;
}

static cplx *to_cplx(const double *d, size_t n) {
  if (!d) return NULL;
  cplx *z = malloc(n * sizeof(cplx));
  for (size_t q = 0; q < n; q++) z[q] = d[2 * q] + I * d[2 * q + 1];
  return z;
}

/* nsteps steps with constant sources and, optionally, laser injection at
 * x_min: the inflow T_r^+, T_th^- of step n at in_rp_d / in_tm_d + n * istride
 * complex elements ([M][nr] each; istride 0: the same every step).  The state
 * is held in the working precision between the steps of one call. */
int ora_step_inflow(int nx, int nr, int M, double h, double dr, double m_a, double g,
                    int flags, double *state_d, const double *jx_d, const double *jr_d,
                    const double *jt_d, const double *sext_d, const double *in_rp_d,
                    const double *in_tm_d, long long istride, int nsteps) {
  if (nx < 4 || nr < 4 || M < 1 || M > 8 || nsteps < 0 || istride < 0) return -1;
  P pp = {nx, nr, M, h, dr, m_a, g, flags, (size_t)M * nx * nr, NULL, NULL};
  const size_t ns = (size_t)N_FIELDS * pp.plane + (size_t)M * nx;
  cplx *S = to_cplx(state_d, ns);
  cplx *jx = to_cplx(jx_d, pp.plane), *jr = to_cplx(jr_d, pp.plane);
  cplx *jt = to_cplx(jt_d, pp.plane), *se = to_cplx(sext_d, pp.plane);
  const size_t nin = (size_t)M * nr;
  int rc = 0;
  for (int n = 0; n < nsteps && rc == 0; n++) {
    cplx *irp = in_rp_d ? to_cplx(in_rp_d + 2 * (size_t)n * istride, nin) : NULL;
    cplx *itm = in_tm_d ? to_cplx(in_tm_d + 2 * (size_t)n * istride, nin) : NULL;
    pp.in_rp = irp;
    pp.in_tm = itm;
    rc = step_once(&pp, S, jx, jr, jt, se);
    free(irp);
    free(itm);
  }
  for (size_t q = 0; q < ns; q++) {
    state_d[2 * q] = (double)RE(S[q]);
    state_d[2 * q + 1] = (double)IM(S[q]);
  }
  free(S); free(jx); free(jr); free(jt); free(se);
  return rc;
}

int ora_step_n(int nx, int nr, int M, double h, double dr, double m_a, double g,
               int flags, double *state_d, const double *jx_d, const double *jr_d,
               const double *jt_d, const double *sext_d, int nsteps) {
  return ora_step_inflow(nx, nr, M, h, dr, m_a, g, flags, state_d, jx_d, jr_d, jt_d, sext_d, NULL, NULL, 0,
                         nsteps);
}

int ora_step(int nx, int nr, int M, double h, double dr, double m_a, double g,
             int flags, double *state_d, const double *jx_d, const double *jr_d,
             const double *jt_d, const double *sext_d) {
  return ora_step_n(nx, nr, M, h, dr, m_a, g, flags, state_d, jx_d, jr_d, jt_d, sext_d, 1);
}

/* ------------------------------------------------------------------------
 * Diagnostics.  Volume integrals use the azimuthal inner product of
 * Eq. fourier_decomp: int_0^{2pi} F G dtheta = 2 pi [F0 G0 + (1/2) sum_{m>0}
 * Re(F_m conj G_m)], and the cell volume 2 pi r dr h, with r_0 replaced by
 * dr/8 on the axis row (the disc of radius dr/2).
 *   out[0] EM energy of group 0, out[1] axion energy, out[2] EM energy of
 *   the regenerated group, out[3] int (E0.E1 + B0.B1) dV.
 *   prof[i] (optional, length nx): U(x_i) = int (1/2)(|E_perp|^2 + |B_perp|^2) dA
 *   (Sec. 4.1), per unit length.
 * ---------------------------------------------------------------------- */
static inline double wmode(int m) { return m == 0 ? 1.0 : 0.5; }
static inline double r_star(const P *p, int j) { return j == 0 ? p->dr / 8.0 : j * p->dr; }

static double em_energy(const P *p, const cplx *S, int g0, double *prof) {
  const cplx *Trp = fld((cplx *)S, p, g0), *Trm = fld((cplx *)S, p, g0 + 1);
  const cplx *Ttp = fld((cplx *)S, p, g0 + 2), *Ttm = fld((cplx *)S, p, g0 + 3);
  const cplx *Ex = fld((cplx *)S, p, g0 + 4), *Bx = fld((cplx *)S, p, g0 + 5);
  const double tpi = 2.0 * 3.14159265358979323846;
  double tot = 0;
  for (int i = 0; i < p->nx; i++) {
    double col = 0, lon = 0;
    for (int m = 0; m < p->M; m++)
      for (int j = 0; j < p->nr; j++) {
        size_t q = ix(p, m, i, j);
        cplx er = 0.5 * (Trp[q] + Trm[q]), bt = 0.5 * (Trp[q] - Trm[q]);
        cplx et = 0.5 * (Ttp[q] + Ttm[q]), br = 0.5 * (Ttp[q] - Ttm[q]);
        double w = wmode(m);
        col += w * (r_half(p, j) * (RE(er * CONJ(er)) + RE(bt * CONJ(bt))) +
                    r_star(p, j) * (RE(et * CONJ(et)) + RE(br * CONJ(br))));
        lon += w * (r_star(p, j) * RE(Ex[q] * CONJ(Ex[q])) +
                    r_half(p, j) * RE(Bx[q] * CONJ(Bx[q])));
      }
    if (prof) prof[i] = 0.5 * tpi * p->dr * col;
    tot += 0.5 * tpi * p->dr * p->h * (col + lon);
  }
  return tot;
}

int ora_diagnostics(int nx, int nr, int M, double h, double dr, double m_a, double g,
                    int flags, const double *state_d, double *out, double *prof) {
  P pp = {nx, nr, M, h, dr, m_a, g, flags, (size_t)M * nx * nr};
  const P *p = &pp;
  cplx *S = to_cplx(state_d, (size_t)N_FIELDS * pp.plane + (size_t)M * nx);
  const double tpi = 2.0 * 3.14159265358979323846;
  out[0] = em_energy(p, S, F_TRP, prof);
  out[2] = em_energy(p, S, F_TRP1, NULL);
  const cplx *phi = fld((cplx *)S, p, F_PHI), *Tap = fld((cplx *)S, p, F_TAP),
             *Tam = fld((cplx *)S, p, F_TAM);
  double ua = 0;
  for (int m = 0; m < M; m++)
    for (int i = 0; i < nx; i++)
      for (int j = 0; j < nr; j++) {
        size_t q = ix(p, m, i, j);
        double w = wmode(m), rh = r_half(p, j);
        /* (1/2)(|T_a^+|^2 + |T_a^-|^2) = |d_t phi|^2 + |d_x phi|^2 (Eq. T_axion_def) */
        ua += w * rh * 0.5 * (RE(Tap[q] * CONJ(Tap[q])) + RE(Tam[q] * CONJ(Tam[q])));
        ua += w * rh * ((double)(m * m) / (rh * rh) + m_a * m_a) * RE(phi[q] * CONJ(phi[q]));
        if (j > 0) {
          cplx d = (phi[q] - phi[ix(p, m, i, j - 1)]) / dr;
          ua += w * r_int(p, j) * RE(d * CONJ(d));
        }
      }
  out[1] = 0.5 * tpi * dr * h * ua;
  double cr = 0;
  for (int m = 0; m < M; m++)
    for (int i = 0; i < nx; i++)
      for (int j = 0; j < nr; j++) {
        size_t q = ix(p, m, i, j);
        double w = wmode(m);
        const cplx *a = S, *b = S;
        cplx er0 = 0.5 * (fld((cplx *)a, p, F_TRP)[q] + fld((cplx *)a, p, F_TRM)[q]);
        cplx bt0 = 0.5 * (fld((cplx *)a, p, F_TRP)[q] - fld((cplx *)a, p, F_TRM)[q]);
        cplx et0 = 0.5 * (fld((cplx *)a, p, F_TTP)[q] + fld((cplx *)a, p, F_TTM)[q]);
        cplx br0 = 0.5 * (fld((cplx *)a, p, F_TTP)[q] - fld((cplx *)a, p, F_TTM)[q]);
        cplx er1 = 0.5 * (fld((cplx *)b, p, F_TRP1)[q] + fld((cplx *)b, p, F_TRM1)[q]);
        cplx bt1 = 0.5 * (fld((cplx *)b, p, F_TRP1)[q] - fld((cplx *)b, p, F_TRM1)[q]);
        cplx et1 = 0.5 * (fld((cplx *)b, p, F_TTP1)[q] + fld((cplx *)b, p, F_TTM1)[q]);
        cplx br1 = 0.5 * (fld((cplx *)b, p, F_TTP1)[q] - fld((cplx *)b, p, F_TTM1)[q]);
        cplx ex0 = fld((cplx *)a, p, F_EX)[q], ex1 = fld((cplx *)b, p, F_EX1)[q];
        cplx bx0 = fld((cplx *)a, p, F_BX)[q], bx1 = fld((cplx *)b, p, F_BX1)[q];
        cr += w * (r_half(p, j) * RE(er0 * CONJ(er1) + bt0 * CONJ(bt1)) +
                   r_star(p, j) * RE(et0 * CONJ(et1) + br0 * CONJ(br1)) +
                   r_star(p, j) * RE(ex0 * CONJ(ex1)) + r_half(p, j) * RE(bx0 * CONJ(bx1)));
      }
  out[3] = tpi * dr * h * cr;
  free(S);
  return 0;
}
