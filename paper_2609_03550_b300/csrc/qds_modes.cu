// qds_modes.cu -- qds_mode_products(): the products of two fields of many
// retained azimuthal modes at many points, sum_p w_p C_m{A_p, B_p}, the form
// of the axion source S_a (Eqs. source_mode_zero/_m) and of the axion current
// j_a (Eqs. jax/jar/jat_mode).  Two methods (Sec. 3.3):
//   direct:  the convolution sums of Eq. mode_convolution, O(M^2) per point;
//   theta:   each field sampled on N angles by an FFT of its zero-padded mode
//            vector (F(theta_s) = Re sum_k F^(k) e^{-i k theta_s}, Eq.
//            fourier_decomp), the products summed over the pairs pointwise,
//            projected back by one more FFT (C_m = (2/N) sum_s P_s e^{i m
//            theta_s}, halved for m = 0); N the power of two >= 3M - 2, the
//            fewest angles that leave the retained modes free of aliasing.
// One warp per point; lanes over the output modes (direct) or over the
// butterflies of a radix-2 FFT in shared memory (theta).
#include <cuda_runtime.h>

#include <cstring>
#include <string>

#include "../../include/qds.h"
#include "qds_common.cuh"

using namespace qds;

// defined in qds_api.cu
void qds_internal_set_error(const std::string &m);

namespace {

constexpr int kMaxModes = 64;
constexpr int kMaxPairs = 4;
constexpr int kWarps = 4;  // points (warps) per block

struct Weights {
  double w[kMaxPairs];
};

int fail_m(int code, const std::string &m) {
  qds_internal_set_error(m);
  return code;
}

// the angles of the theta grid: a power of two, at least 3M - 2 (and 2)
int theta_points(int M) {
  int n = 2;
  while (n < 3 * M - 2) n <<= 1;
  return n;
}

template <class R>
__device__ __forceinline__ C<R> cmul(C<R> a, C<R> b) {
  return mk<R>(a.re * b.re - a.im * b.im, a.re * b.im + a.im * b.re);
}
template <class R>
__device__ __forceinline__ C<R> cmul_cb(C<R> a, C<R> b) {  // a conj(b)
  return mk<R>(a.re * b.re + a.im * b.im, a.im * b.re - a.re * b.im);
}

// ---------------------------------------------------------------------------
// Direct: lane m (and m + 32) of the point's warp forms output mode m from
// the point's mode vectors in shared memory.
// ---------------------------------------------------------------------------
template <class R>
__global__ void __launch_bounds__(32 * kWarps) products_direct(int M, int npts, int npairs, const C<R> *__restrict__ A,
                                                              const C<R> *__restrict__ B, Weights wt, C<R> *out) {
  __shared__ C<R> sa[kWarps][kMaxPairs][kMaxModes], sb[kWarps][kMaxPairs][kMaxModes];
  const int wp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  for (int q = blockIdx.x * kWarps + wp; q < npts; q += gridDim.x * kWarps) {
    for (int p = 0; p < npairs; p++)
      for (int k = lane; k < M; k += 32) {
        sa[wp][p][k] = A[((size_t)p * M + k) * npts + q];
        sb[wp][p][k] = B[((size_t)p * M + k) * npts + q];
      }
    __syncwarp();
    for (int m = lane; m < M; m += 32) {
      C<R> s = zero<R>();
      for (int p = 0; p < npairs; p++) {
        const C<R> *a = sa[wp][p], *b = sb[wp][p];
        C<R> t = zero<R>();
        if (m == 0) {
          t = cmul(a[0], b[0]);
          R h = R(0);
          for (int k = 1; k < M; k++) h += a[k].re * b[k].re + a[k].im * b[k].im;
          t.re += R(0.5) * h;
        } else {
          for (int k = 0; k <= m && k < M; k++)
            if (m - k < M) t += cmul(a[k], b[m - k]);            // k + l = m
          for (int l = 0; l + m < M; l++) t += cmul_cb(a[l + m], b[l]);  // k - l = m
          for (int k = 0; k + m < M; k++) t += cmul_cb(b[k + m], a[k]);  // l - k = m
          t = R(0.5) * t;
        }
        s += R(p == 0 ? wt.w[0] : p == 1 ? wt.w[1] : p == 2 ? wt.w[2] : wt.w[3]) * t;
      }
      out[(size_t)m * npts + q] = s;
    }
    __syncwarp();
  }
}

// ---------------------------------------------------------------------------
// Theta grid: radix-2 decimation-in-time FFT of N points held in shared
// memory by one warp, X_s = sum_k x_k e^{-2 pi i k s / N}; tw[t] = e^{-2 pi i t/N}.
// ---------------------------------------------------------------------------
__device__ __forceinline__ int bitrev(int i, int logn) { return (int)(__brev((unsigned)i) >> (32 - logn)); }

template <class R>
__device__ void warp_fft(C<R> *X, const C<R> *tw, int N, int logn, int lane) {
  for (int len = 2; len <= N; len <<= 1) {
    const int half = len >> 1, tstep = N / len;
    for (int b = lane; b < (N >> 1); b += 32) {
      const int pos = b & (half - 1), i0 = (b - pos) * 2 + pos, i1 = i0 + half;
      const C<R> u = X[i0], v = cmul(X[i1], tw[pos * tstep]);
      X[i0] = u + v;
      X[i1] = u - v;
    }
    __syncwarp();
  }
}

template <class R>
__global__ void __launch_bounds__(32 * kWarps) products_theta(int M, int npts, int npairs, int N, int logn,
                                                             const C<R> *__restrict__ A, const C<R> *__restrict__ B,
                                                             Weights wt, C<R> *out) {
  extern __shared__ __align__(16) unsigned char smraw[];
  C<R> *tw = reinterpret_cast<C<R> *>(smraw);        // N/2 twiddles
  C<R> *X0 = tw + N / 2;                             // kWarps transform buffers of N
  const int wp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  for (int t = threadIdx.x; t < N / 2; t += blockDim.x) {
    // e^{-2 pi i t / N}, formed in FP64 and rounded to R
    double sn, cs;
    sincospi(-2.0 * (double)t / (double)N, &sn, &cs);
    tw[t] = mk<R>((R)cs, (R)sn);
  }
  __syncthreads();
  C<R> *X = X0 + (size_t)wp * N;
  constexpr int kPer = 8;  // samples per lane (N <= 256)
  for (int q = blockIdx.x * kWarps + wp; q < npts; q += gridDim.x * kWarps) {
    R P[kPer];
#pragma unroll
    for (int t = 0; t < kPer; t++) P[t] = R(0);
    for (int p = 0; p < npairs; p++) {
      R fa[kPer];
      const R wp_ = R(p == 0 ? wt.w[0] : p == 1 ? wt.w[1] : p == 2 ? wt.w[2] : wt.w[3]);
      for (int side = 0; side < 2; side++) {
        const C<R> *src = (side == 0 ? A : B) + (size_t)p * M * npts + q;
        for (int i = lane; i < N; i += 32) X[bitrev(i, logn)] = i < M ? src[(size_t)i * npts] : zero<R>();
        __syncwarp();
        warp_fft(X, tw, N, logn, lane);
        // F(theta_s) = Re X_s (sample s = lane + 32 t of this lane)
#pragma unroll
        for (int t = 0; t < kPer; t++) {
          const int s = lane + 32 * t;
          if (s < N) {
            if (side == 0) fa[t] = X[s].re;
            else P[t] += wp_ * fa[t] * X[s].re;
          }
        }
        __syncwarp();
      }
    }
#pragma unroll
    for (int t = 0; t < kPer; t++) {
      const int s = lane + 32 * t;
      if (s < N) X[bitrev(s, logn)] = mk<R>(P[t], R(0));
    }
    __syncwarp();
    warp_fft(X, tw, N, logn, lane);
    // C_m = (2/N) conj(Y_m), halved for m = 0
    for (int m = lane; m < M; m += 32) {
      const R f = (m == 0 ? R(1) : R(2)) / R(N);
      out[(size_t)m * npts + q] = mk<R>(f * X[m].re, -f * X[m].im);
    }
    __syncwarp();
  }
}

template <class R>
int run(int M, int npts, int npairs, const void *A, const void *B, const double *w, void *out, int method,
        cudaStream_t st) {
  Weights wt;
  std::memset(&wt, 0, sizeof wt);
  for (int p = 0; p < npairs; p++) wt.w[p] = w[p];
  const int blocks = (int)std::min<long long>(((long long)npts + kWarps - 1) / kWarps, 148LL * 16);
  if (npts == 0) return QDS_OK;
  if (method == QDS_MODES_DIRECT) {
    products_direct<R><<<blocks, 32 * kWarps, 0, st>>>(M, npts, npairs, (const C<R> *)A, (const C<R> *)B, wt,
                                                      (C<R> *)out);
  } else {
    const int N = theta_points(M);
    int logn = 0;
    while ((1 << logn) < N) logn++;
    const size_t smem = sizeof(C<R>) * (size_t)(N / 2 + kWarps * N);
    products_theta<R><<<blocks, 32 * kWarps, smem, st>>>(M, npts, npairs, N, logn, (const C<R> *)A,
                                                         (const C<R> *)B, wt, (C<R> *)out);
  }
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return fail_m(QDS_ERR_CUDA, std::string("mode products launch: ") + cudaGetErrorString(e));
  return QDS_OK;
}

}  // namespace

extern "C" int qds_mode_products_theta_points(int n_modes) {
  return n_modes >= 1 && n_modes <= kMaxModes ? theta_points(n_modes) : 0;
}

extern "C" int qds_mode_products(int n_modes, int npts, int npairs, const void *a_dev, const void *b_dev,
                                 const double *w_host, void *out_dev, int method, int fp32, void *stream) {
  if (n_modes < 1 || n_modes > kMaxModes) return fail_m(QDS_ERR_INVALID_ARG, "mode products: n_modes must be 1..64");
  if (npairs < 1 || npairs > kMaxPairs) return fail_m(QDS_ERR_INVALID_ARG, "mode products: npairs must be 1..4");
  if (npts < 0) return fail_m(QDS_ERR_INVALID_ARG, "mode products: npts < 0");
  if (!w_host || (npts > 0 && (!a_dev || !b_dev || !out_dev)))
    return fail_m(QDS_ERR_INVALID_ARG, "mode products: NULL argument");
  if (method != QDS_MODES_DIRECT && method != QDS_MODES_THETA)
    return fail_m(QDS_ERR_INVALID_ARG, "mode products: unknown method");
  cudaStream_t st = (cudaStream_t)stream;
  if (fp32) return run<float>(n_modes, npts, npairs, a_dev, b_dev, w_host, out_dev, method, st);
  return run<double>(n_modes, npts, npairs, a_dev, b_dev, w_host, out_dev, method, st);
}
