// Householder QR of a dense complex matrix on the GPU (CUDA, sm_103a, FP64): the least-squares
// solve of the coupled subdomain system (Section 3.5, steps 2(b)-(c): "QR").
//
// A is column-major m x (n + nrhs). For k = 0 .. n-1 the reflector H_k = I - tau_k v_k v_k^H
// (v_k(k) = 1, v_k zero above k) maps column k below the diagonal onto beta_k e_k with beta_k
// real, and H_k^H is applied to the columns right of k, including the nrhs right-hand sides:
// on return the upper triangle of the first n columns is R, the reflectors sit below it, tau
// holds tau_k, and the last nrhs columns hold Q^H b. The construction follows the textbook
// Householder method: with x = A(k:m, k), alpha = x(0),
//   beta = -sign(Re alpha) ||x||,  tau = (beta - alpha) / beta,  v = x / (alpha - beta), v(0) = 1.
// A batch of equal-shaped matrices (stride elements apart) is factored together: launch y
// index = matrix. One launch per column: block b applies H_k^H to column k+1+b (w = v^H a, a -= conj(tau) v w)
// and block 0, which holds column k+1, then forms the next reflector from it. Reductions run in
// a fixed order (deterministic).
#include "kernels_common.cuh"

#include "mdp.h"

namespace mdp {
namespace {

constexpr int kQrThreads = 256;

__device__ __forceinline__ double block_sum_qr(double v, double *sh) {
  const int t = threadIdx.x;
  sh[t] = v;
  __syncthreads();
  for (int s = kQrThreads / 2; s > 0; s >>= 1) {
    if (t < s) sh[t] += sh[t + s];
    __syncthreads();
  }
  const double r = sh[0];
  __syncthreads();
  return r;
}

// The reflector of column k (in place) and tau_k; one block.
__device__ void qr_reflector(int m, int k, double2 *A, long long lda, double2 *tau, double *sh) {
  double2 *x = A + (long long)k * lda;
  double s = 0.0;
  for (int i = k + 1 + threadIdx.x; i < m; i += kQrThreads) s = fma(x[i].x, x[i].x, fma(x[i].y, x[i].y, s));
  const double xn2 = block_sum_qr(s, sh);   // ||x(1:)||^2
  const double2 a = x[k];
  if (xn2 == 0.0 && a.y == 0.0) {           // already of the form beta e_k: H = I
    if (threadIdx.x == 0) tau[k] = make_double2(0.0, 0.0);
    return;
  }
  const double nrm = sqrt(fma(a.x, a.x, fma(a.y, a.y, xn2)));
  const double beta = a.x >= 0.0 ? -nrm : nrm;
  // scale = 1 / (alpha - beta)
  const double dr = a.x - beta, di = a.y, den = fma(dr, dr, di * di);
  const double sr = dr / den, si = -di / den;
  for (int i = k + 1 + threadIdx.x; i < m; i += kQrThreads) {
    const double2 v = x[i];
    x[i] = make_double2(fma(v.x, sr, -v.y * si), fma(v.x, si, v.y * sr));
  }
  if (threadIdx.x == 0) {
    tau[k] = make_double2((beta - a.x) / beta, -a.y / beta);
    x[k] = make_double2(beta, 0.0);
  }
}

__global__ void __launch_bounds__(kQrThreads) k_qr_first(int m, int n, double2 *A, long long lda, long long stride,
                                                          double2 *tau) {
  __shared__ double sh[kQrThreads];
  qr_reflector(m, 0, A + (long long)blockIdx.y * stride, lda, tau + (long long)blockIdx.y * n, sh);
}

// Step k: column k+1+blockIdx.x gets w = v^H a (v(k) = 1), a -= conj(tau) v w; block 0 then
// forms the reflector of column k+1 for step k+1 (n: the number of columns to factor).
__global__ void __launch_bounds__(kQrThreads) k_qr_step(int m, int n, int k, double2 *A, long long lda,
                                                         long long stride, double2 *tau) {
  __shared__ double sh[kQrThreads];
  A += (long long)blockIdx.y * stride;   // matrix blockIdx.y of the batch
  tau += (long long)blockIdx.y * n;
  const double2 t = tau[k];
  const double2 *v = A + (long long)k * lda;
  double2 *a = A + (long long)(k + 1 + blockIdx.x) * lda;
  if (t.x != 0.0 || t.y != 0.0) {
    double wr = 0.0, wi = 0.0;
    for (int i = k + threadIdx.x; i < m; i += kQrThreads) {
      const double2 vi = i == k ? make_double2(1.0, 0.0) : v[i];
      const double2 ai = a[i];
      wr = fma(vi.x, ai.x, fma(vi.y, ai.y, wr));      // conj(v) a
      wi = fma(vi.x, ai.y, fma(-vi.y, ai.x, wi));
    }
    wr = block_sum_qr(wr, sh);
    wi = block_sum_qr(wi, sh);
    const double cr = fma(t.x, wr, t.y * wi), ci = fma(t.x, wi, -t.y * wr);   // conj(tau) w
    for (int i = k + threadIdx.x; i < m; i += kQrThreads) {
      const double2 vi = i == k ? make_double2(1.0, 0.0) : v[i];
      double2 ai = a[i];
      ai.x -= fma(vi.x, cr, -vi.y * ci);
      ai.y -= fma(vi.x, ci, vi.y * cr);
      a[i] = ai;
    }
  }
  if (blockIdx.x == 0 && k + 1 < n) {
    __syncthreads();   // the column's updates by every thread precede its reflector
    qr_reflector(m, k + 1, A, lda, tau, sh);
  }
}

}  // namespace
}  // namespace mdp

extern "C" mdp_status mdp_householder_qr_batched(int batch, int m, int n, int nrhs, mdp_c64 *A, long long lda,
                                                 long long stride, mdp_c64 *tau, void *cuda_stream) {
  if (batch < 1 || batch > 65535 || m < 1 || n < 1 || n > m || nrhs < 0 || !A || !tau || lda < m ||
      (batch > 1 && stride < lda * (long long)(n + nrhs)))
    return MDP_ERR_ARG;
  cudaStream_t st = (cudaStream_t)cuda_stream;
  double2 *a = reinterpret_cast<double2 *>(A);
  double2 *t = reinterpret_cast<double2 *>(tau);
  mdp::k_qr_first<<<dim3(1, batch), mdp::kQrThreads, 0, st>>>(m, n, a, lda, stride, t);
  for (int k = 0; k < n; ++k) {
    const int ncol = n + nrhs - k - 1;
    if (ncol > 0) mdp::k_qr_step<<<dim3(ncol, batch), mdp::kQrThreads, 0, st>>>(m, n, k, a, lda, stride, t);
  }
  return cudaGetLastError() == cudaSuccess ? MDP_OK : MDP_ERR_CUDA;
}

extern "C" mdp_status mdp_householder_qr(int m, int n, int nrhs, mdp_c64 *A, long long lda, mdp_c64 *tau,
                                         void *cuda_stream) {
  return mdp_householder_qr_batched(1, m, n, nrhs, A, lda, 0, tau, cuda_stream);
}
