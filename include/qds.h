/*
 * qds.h -- C ABI of the B300 QDS field-step library (libqds.so).
 *
 * One step advances, for every retained azimuthal mode m (Sec. 2, Eq.
 * fourier_decomp), the quasi-cylindrical direction-splitting (QDS) Maxwell
 * solve of Sec. 2.1 (characteristic shift of T_r^+-, T_theta^+- by exactly
 * one cell with c dt = dx, Eqs. Trp/Trm/Ttp/Ttm_update; leapfrog of E_x, B_x,
 * Eq. Ex_update; axis rules of Sec. 2.3; open boundaries of Sec. 3.2), the
 * Klein-Gordon axion transport of Sec. 2.2 (Eqs. Ta_plus_update,
 * Ta_minus_update, phi_update, mode convolution Eq. mode_convolution) and the
 * axion-regenerated fields (Eqs. jax_mode, jar_mode, jat_mode), driven by
 * given current arrays.  Normalised units: c = eps0 = mu0 = hbar = 1.
 *
 * Memory: the caller allocates (and owns) the field-state buffer of
 * qds_state_bytes() bytes, 256-byte aligned, and any source arrays; all of
 * them are device pointers.  The handle owns only small descriptor tables
 * and captured CUDA graphs, released by qds_free().
 *
 * Layouts: a "complex plane set" [M][nx][nr] stores mode m, x index i and
 * radial index j at ((m*nx + i)*nr + j), each element an interleaved
 * (re, im) pair of the working precision (float for QDS_FP32, else double).
 * Inside the library's state buffer the row stride is nr rounded up to even
 * in FP32 (every column starts on a 16-byte boundary for the bulk copies);
 * callers never see that layout (qds_set_state / qds_get_state convert).
 * Staggering: T_r at (x_i, r_{j+1/2}), T_theta at (x_i, r_j), E_x at
 * (x_{i+1/2}, r_j), B_x and phi at (x_{i+1/2}, r_{j+1/2}), T_a at
 * (x_i, r_{j+1/2}); r_j = j dr.  Faces i = 0..nx-2 are real (nx-1 is held
 * at zero unless x is periodic).
 *
 * Canonical state (qds_set_state / qds_get_state): complex128 planes
 *   fields[15][M][nx][nr] in the order Trp Trm Ttp Ttm Ex Bx phi Tap Tam
 *   Trp1 Trm1 Ttp1 Ttm1 Ex1 Bx1, then phi_prev[M][nx]
 * (phi on the outermost half row one step back), in physical units and
 * window order whatever the working precision and ring offset.
 *
 * Errors: every int-returning call returns QDS_OK (0) or a QDS_ERR_* code
 * and sets a message readable with qds_last_error() (thread-local).  No call
 * aborts the process or traps the device.  Kernel launches are asynchronous:
 * a later call on the same stream (or a stream synchronise) reports faults.
 */
#ifndef QDS_H
#define QDS_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define QDS_OK 0
#define QDS_ERR_INVALID_ARG 1
#define QDS_ERR_CUDA 2
#define QDS_ERR_NONFINITE 3   /* a NaN or Inf reached the state (step kernels, energies) */
#define QDS_ERR_TIMEOUT 4     /* a bounded device wait (bulk copy of a step kernel) ran out */
#define QDS_ERR_UNSUPPORTED 5

/* flags */
#define QDS_AXION 1u          /* advance phi and T_a (Sec. 2.2)                        */
#define QDS_AREM 2u           /* advance the axion-regenerated fields (needs QDS_AXION) */
#define QDS_MOVING_WINDOW 4u  /* box moves one cell per step (ring offset, zero inflow)  */
#define QDS_X_PERIODIC 8u     /* periodic x (test mode)                                 */
#define QDS_R_CLOSED 16u      /* conducting wall / Neumann axion at r = nr dr (test)    */
#define QDS_FP32 32u          /* FP32 storage and arithmetic (implies QDS_SCALE_G)      */
#define QDS_SCALE_G 64u       /* store phi/g and (E1, B1)/g^2 internally                */

/* The statement of one solve (Sec. 2): grid, retained modes, steps, axion. */
typedef struct qds_params {
  int32_t nx;              /* cells along x (>= 8)                                    */
  int32_t nr;              /* radial rows (>= 4): integer rows 0..nr-1, half rows 1/2..nr-1/2 */
  int32_t n_modes;         /* retained modes M (1..4)                                 */
  const int32_t *modes;    /* host array {0, 1, ..., M-1} or NULL                     */
  double dx, dr, dt;       /* c dt must equal dx; stability needs
                              dr >= dx max(1.5, M - 3/4)(1 + dx m_a)                  */
  double omega0;           /* laser frequency used only by callers' normalisations   */
  double m_a;              /* axion mass (normalised wavenumber), dx m_a <= 1         */
  double g;                /* axion-photon coupling g_{a gamma gamma} (normalised)    */
  uint32_t flags;          /* QDS_* bits                                              */
} qds_params;

/* Per-step drive, device pointers in the working precision, complex plane
 * sets [M][nx][nr] at native positions; any may be NULL (zero).
 *   jx  at (x_{i+1/2}, r_j,     t^n)
 *   jr  at (x_i,       r_{j+1/2}, t^{n+1/2})
 *   jth at (x_i,       r_j,     t^{n+1/2})
 *   s_ext: additive axion source at (x_{i+1/2}, r_{j+1/2}, t^n) (test hook)
 * They must stay valid until the stream has executed the steps that use them.
 * Sources are taken in window order (slot = window index); with a moving
 * window the caller provides them in window coordinates each step. */
typedef struct qds_sources {
  const void *jx, *jr, *jth, *s_ext;
} qds_sources;

typedef struct qds_handle qds_handle;

/* Bytes of caller-owned state for one solve (two ping-pong copies of the
 * 15 planes + phi_prev, and four scratch planes, in the working precision);
 * 0 if params are invalid. */
size_t qds_state_bytes(const qds_params *p);

/* Create a solver bound to state_dev (>= qds_state_bytes, 256-byte aligned).
 * Returns QDS_ERR_INVALID_ARG for an inconsistent or unstable statement
 * (c dt != dx, dr below the stability bound, bad mode list, ...). */
int qds_create(const qds_params *p, void *state_dev, size_t bytes, qds_handle **out);

/* Import the canonical complex128 state (device pointer) and reset the step
 * counter; asynchronous on stream (a cudaStream_t, NULL = default stream). */
int qds_set_state(qds_handle *h, const void *src_dev, void *stream);

/* Export the canonical complex128 state (device pointer), asynchronous. */
int qds_get_state(qds_handle *h, void *dst_dev, void *stream);

/* Advance nsteps steps; calls of >= 16 steps replay a captured CUDA graph.
 * src != NULL sets the sources of every instance for this and later calls
 * to these arrays, the same every step (all pointers NULL: no sources; a
 * batch takes only that, its sources are set per instance); src == NULL
 * keeps the sources set before (qds_set_sources_i or an earlier call).
 * Asynchronous on stream: a batch with several mode counts runs each mode
 * count's kernels on a stream of the handle, forked from and joined back to
 * `stream` by events, so the call is ordered on `stream` like a single
 * launch. */
int qds_step(qds_handle *h, const qds_sources *src, int nsteps, void *stream);

/* Sources of instance i for the following qds_step calls (src NULL: none).
 * Step k of a call (k = 0, 1, ...) reads every array of src advanced by
 * k * stride elements (complex values of the working precision; stride 0:
 * the same arrays every step), so that a call of n steps can take n steps
 * of a driven run at once: with stride M*nx*nr the arrays are [n][M][nx][nr].
 * The arrays must stay valid until the stream has executed those steps.
 * Uploads the descriptor (synchronises stream). */
int qds_set_sources_i(qds_handle *h, int i, const qds_sources *src, long long stride, void *stream);

/* Laser injection at x_min (Sec. 4.1 injects its vacuum pulse through the
 * boundary; Eq. em_x_open sets the inflow characteristics to zero there):
 * for the following qds_step calls the exterior cell behind x_min holds the
 * inflow T_r^+ = E_r + B_theta (tr_plus_dev) and T_theta^- = E_theta - B_r
 * (tth_minus_dev) of the EM field at time n, so that the shift carries them
 * into cell 0 at step n -> n+1 (the outgoing T_r^-, T_theta^+ and all other
 * fields stay zero outside; the axion and the regenerated field are not
 * injected).  Arrays: [M][nr] complex values of the working precision
 * (device), physical variables; step k of a call reads them advanced by
 * k * stride elements (stride 0: the same every step; M*nr: [n][M][nr]).
 * NULL for either array gives zero inflow for it; both NULL restores the
 * open boundary.  Open x only (QDS_X_PERIODIC: QDS_ERR_INVALID_ARG).  The
 * arrays must stay valid until the stream has executed those steps.
 * Uploads the descriptor (synchronises stream). */
int qds_set_inflow_i(qds_handle *h, int i, const void *tr_plus_dev, const void *tth_minus_dev, long long stride,
                     void *stream);

/* Energies into out_host[4] = {EM energy, axion energy, regenerated EM
 * energy, int (E0.E1 + B0.B1) dV} (mode-weighted volume integrals, FP64,
 * compensated sums); if profile_dev is non-NULL (device, nx doubles) also the
 * transverse energy per unit length U(x) of Sec. 4.1.  Synchronises stream. */
int qds_diagnostics(qds_handle *h, double *out_host, double *profile_dev, void *stream);

/* Batched solves: n independent statements (uneven grids and mode counts,
 * one precision) advanced together, one launch per mode count per step.
 * Instance i owns a contiguous block of the state arena in order. */
size_t qds_batch_state_bytes(int n, const qds_params *p);
int qds_batch_create(int n, const qds_params *p, void *state_dev, size_t bytes, qds_handle **out);
int qds_set_state_i(qds_handle *h, int i, const void *src_dev, void *stream);
int qds_get_state_i(qds_handle *h, int i, void *dst_dev, void *stream);
int qds_diagnostics_i(qds_handle *h, int i, double *out_host, double *profile_dev, void *stream);
int qds_num_instances(const qds_handle *h);
/* The four energies of every instance into out_dev[4*i .. 4*i+3] (device,
 * n_inst*4 doubles) in two launches; asynchronous on stream. */
int qds_diagnostics_all(qds_handle *h, double *out_dev, void *stream);

/* Step implementation (both give the same results to rounding):
 *   QDS_STEP_DEFAULT  QDS_STEP_FLAT (the faster of the two measured on the
 *                     batched scan);
 *   QDS_STEP_FLAT     one grid-wide pass per stage group (leapfrog, axion
 *                     source, shift + phi, axion current + regenerated
 *                     leapfrog, regenerated shift, window zeroing), one
 *                     point per thread over flat ranges of 256 points,
 *                     intermediates in the new state and scratch planes;
 *   QDS_STEP_MARCH    two x-marching kernels per mode count: each CTA walks
 *                     a band of rows (all modes, one thread per row and
 *                     mode) along x, the old state arriving column by
 *                     column in a shared-memory ring by bulk tensor copies,
 *                     two columns ahead; the first kernel advances the EM
 *                     field and the axion and writes j_a (one extra warp
 *                     forms the outer half row's boundary values), the
 *                     second the axion-regenerated field.
 * Changing the mode drops the captured graphs. */
#define QDS_STEP_DEFAULT 0
#define QDS_STEP_FLAT 1
#define QDS_STEP_MARCH 2
int qds_set_step_mode(qds_handle *h, int mode);
/* Kernel launches of one step in the current mode (0 for a NULL handle). */
int qds_step_launches(const qds_handle *h);

/* Work split of QDS_STEP_MARCH (the autotuner's knobs): rows = ring rows
 * per CTA including the radial halo, 64 or 32 in FP32 and 32 in FP64 (a
 * request is rounded down to one of these, at least 32; 0 = 64 in FP32),
 * cols = window columns per CTA (>= 4; 0 = 128).  qds_get_tile reports the
 * rows of the first kernel of the first mode count, the columns, the CTAs of
 * one step and that kernel's shared memory in bytes. */
int qds_set_tile(qds_handle *h, int rows, int cols);
int qds_get_tile(qds_handle *h, int *rows, int *cols, int *ntiles, int *smem_bytes);

/* Device error state since the last qds_set_state: QDS_OK, QDS_ERR_TIMEOUT
 * or QDS_ERR_NONFINITE (the step kernels flag a non-finite T_r^+ or T_a^+
 * they store; the energy reductions flag a non-finite energy).  Synchronises
 * stream.  qds_diagnostics returns the same codes. */
int qds_status(qds_handle *h, void *stream);

/* Test hook for the failure path: with on != 0 every x-marching CTA of the
 * following steps withholds its first bulk copy, so that its bounded wait
 * on that column runs out (about a second); the CTA then sets the timeout
 * bit, lets its other copies land and exits, and qds_status reports
 * QDS_ERR_TIMEOUT.  The fields of those steps are not valid.  on = 0
 * restores normal operation (qds_set_state clears the error bits).
 * Asynchronous on stream. */
int qds_test_withhold_copy(qds_handle *h, int on, void *stream);

void qds_free(qds_handle *h);
const char *qds_last_error(void);

/* ---------------------------------------------------------------------------
 * Mode products for many retained modes (Sec. 3.3).  For npts points:
 *   out[m][q] = sum_{p < npairs} w[p] C_m{A_p[.][q], B_p[.][q]},  m < n_modes,
 * C_m the mode convolution of Eq. mode_convolution (the form of the axion
 * source, Eqs. source_mode_zero/_m, and of the axion current, Eqs.
 * jax/jar/jat_mode; w folds their signs and halves).  method:
 *   QDS_MODES_DIRECT  the convolution sums, O(n_modes^2) per point;
 *   QDS_MODES_THETA   the theta-grid procedure of Sec. 3.3: every field
 *                     sampled on N angles by an FFT of its mode vector, the
 *                     products summed over the pairs pointwise, projected
 *                     back by one more FFT; N the power of two >= 3 n_modes
 *                     - 2 (qds_mode_products_theta_points), the fewest angles
 *                     that leave the retained modes free of aliasing.  Exact
 *                     for real fields (real m = 0 components).
 * a_dev, b_dev: [npairs][n_modes][npts], out_dev: [n_modes][npts], complex
 * device arrays (complex64 if fp32 else complex128); w_host: npairs doubles.
 * 1 <= n_modes <= 64, 1 <= npairs <= 4.  Asynchronous on stream. */
#define QDS_MODES_DIRECT 0
#define QDS_MODES_THETA 1
int qds_mode_products(int n_modes, int npts, int npairs, const void *a_dev, const void *b_dev, const double *w_host,
                      void *out_dev, int method, int fp32, void *stream);
int qds_mode_products_theta_points(int n_modes);

/* ---------------------------------------------------------------------------
 * Synthetic per-step currents of the driven workloads (input generation, not
 * part of the scheme), for the `count` steps step .. step + count - 1:
 * j_x, j_r, j_theta [count][n_modes][nx][nr] (interleaved complex, FP32 or
 * FP64 per fp32) receive uniform noise in [-amp, amp) on the real and
 * imaginary parts of every mode and cell (m = 0 real), and j_x of m = 0 also
 * the bunch bunch_dev [nx][nr] (FP64, may be NULL).  The noise of element e
 * (components, then modes, x and r) of step n is SplitMix64 (Steele, Lea and
 * Flood, OOPSLA 2014) of a key made from seed and n, plus 2e (real) and
 * 2e + 1 (imaginary); with u its top 24 bits the value is the FP32 number
 * (float)amp * (u 2^-23 - 1), the same in FP32 and FP64 runs; the bunch is
 * added in FP64 and the sum rounded once.  Any step redraws alone with the
 * same values.  Asynchronous on stream; returns
 * QDS_ERR_INVALID_ARG for bad sizes or NULL outputs. */
int qds_bunch_currents(int n_modes, int nx, int nr, unsigned long long seed, unsigned long long step, int count,
                       double amp, const double *bunch_dev, void *jx_dev, void *jr_dev, void *jth_dev, int fp32,
                       void *stream);

/* ---------------------------------------------------------------------------
 * Adjoint (transpose) of one step of the EM group and the axion (Sec. 2;
 * the transpose of the +x transport shift is the -x shift).  For a real
 * functional L of the state the adjoint of a complex value z is
 * dL/dRe z + i dL/dIm z.  The regenerated group does not feed back into the
 * EM fields or the axion, so for functionals of those it has a zero adjoint
 * and its slots in the result are zero.
 *
 * fwd_state_dev: the forward state of instance i at the START of the step
 *   (canonical complex128 layout of qds_set_state, physical variables: what
 *   qds_get_state_i returned then).  Read only.
 * adj_state_dev: on entry the adjoint of the state after the step, on exit
 *   the adjoint of the state before it (same layout, complex128).
 * src: the sources that step used (jx and jth enter the linearisation,
 *   s_ext enters dL/dg; working precision, as for qds_step); may be NULL.
 * work_dev: caller-owned scratch of >= qds_adjoint_work_bytes(h, i) bytes,
 *   256-byte aligned.
 * dLdg_dev: device double to which dL/dg of this step is ADDED (may be NULL).
 * Open boundaries only (QDS_X_PERIODIC / QDS_R_CLOSED: QDS_ERR_UNSUPPORTED);
 * needs QDS_AXION.  Runs in the handle's precision (QDS_FP32: complex64
 * arithmetic, results widened to complex128).  Asynchronous on stream. */
size_t qds_adjoint_work_bytes(const qds_handle *h, int i);
/* The same transpose without conversions, for the adjoint's
 * checkpoint-and-recompute in the working precision:
 * fwd_working_dev: a working snapshot of instance i (qds_save_working) taken
 *   fwd_step steps after the state import, at the START of the step (its
 *   EM planes are read; working row stride and window offset).
 * fwd_next_dev: the snapshot at the END of the step (fwd_step + 1), or NULL.
 *   Its E_x, B_x planes hold the leapfrog's E_x, B_x^(n+1/2), which the
 *   transpose otherwise recomputes from fwd_working_dev.
 * lam_in_dev / lam_out_dev: the adjoint of the state after / before the step
 *   in the canonical layout of qds_set_state but in the working precision
 *   (complex64 with QDS_FP32, else complex128), physical variables; distinct
 *   buffers.  Every entry of lam_out is written except the regenerated
 *   group's six plane sets, which are left as they are (zero them once).
 * work_dev: >= qds_adjoint_work_bytes_w(h, i) bytes, 256-byte aligned.
 * Otherwise as qds_adjoint_step.  Asynchronous on stream. */
size_t qds_adjoint_work_bytes_w(const qds_handle *h, int i);
int qds_adjoint_step_w(qds_handle *h, int i, const qds_sources *src, const void *fwd_working_dev,
                       const void *fwd_next_dev, unsigned long long fwd_step, const void *lam_in_dev,
                       void *lam_out_dev, void *work_dev, size_t work_bytes, double *dLdg_dev, void *stream);

/* Working snapshots, the checkpoints of the adjoint's recompute (the paper
 * defines no adjoint; these serve qds_adjoint_step_w): the state of instance
 * i as the kernels hold it (working precision, 1/g-scaled axion and
 * regenerated groups in FP32, padded row stride, ring offset of the moving
 * window), qds_working_bytes(h, i) bytes.
 * qds_steps_taken: steps since the last qds_set_state / qds_restore_working
 *   (the host's count of the qds_step calls; it fixes the window offset).
 * qds_save_working: copies the current state into dst_dev (asynchronous);
 *   with bytes < qds_working_bytes only the first bytes (the EM group's six
 *   plane sets, 6 n_modes nx ld elements, lead the state).
 * qds_restore_working: makes a snapshot taken `step` steps after the import
 *   the current state again and sets the step count to `step` (a handle of
 *   one instance; clears the device error bits).  Asynchronous on stream. */
size_t qds_working_bytes(const qds_handle *h, int i);
unsigned long long qds_steps_taken(const qds_handle *h);
int qds_save_working(qds_handle *h, int i, void *dst_dev, size_t bytes, void *stream);
int qds_restore_working(qds_handle *h, const void *src_dev, size_t bytes, unsigned long long step, void *stream);
int qds_adjoint_step(qds_handle *h, int i, const qds_sources *src, const void *fwd_state_dev,
                     void *adj_state_dev, void *work_dev, size_t work_bytes, double *dLdg_dev, void *stream);

/* ---------------------------------------------------------------------------
 * No-allocation step (this entry point has no counterpart in the paper; it
 * serves callers that cannot allocate device memory: code inside runtimes
 * or memory pools that forbid allocation after start-up, plug-ins that must
 * not grow a host application's device footprint, real-time loops where an
 * allocation may stall or fail).
 *
 * Imports the canonical complex128 state state_in_dev, advances it nsteps
 * steps (pass-mode kernels, no sources) and exports it to state_out_dev
 * (which may equal state_in_dev).  work_dev (>= qds_state_bytes(p) bytes,
 * 256-byte aligned, caller-owned) holds the two working copies of the
 * state.  The descriptor, step counter, tile table and the four scratch
 * planes live in one static device array of QDS_NOALLOC_SCRATCH_BYTES
 * bytes that every GPU loading the library holds until exit; a statement
 * whose scratch does not fit returns QDS_ERR_INVALID_ARG.  No cudaMalloc,
 * cudaFree or graph instantiation is made.  The first call on a device
 * looks up the array's device address (cudaGetSymbolAddress) with that
 * device current; make that first call before any stream capture.  All
 * calls share the array: the call rewrites the descriptor and clears the
 * scratch on entry, synchronises the stream once during that set-up, and
 * calls that overlap on the GPU (other streams, other threads) race.
 * ------------------------------------------------------------------------- */
#define QDS_NOALLOC_SCRATCH_BYTES (32u << 20)
int qds_advance_noalloc(const qds_params *p, const void *state_in_dev, void *state_out_dev,
                        void *work_dev, size_t work_bytes, int nsteps, void *stream);

#ifdef __cplusplus
}
#endif

#endif /* QDS_H */
