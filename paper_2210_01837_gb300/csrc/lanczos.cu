// Brownian increments g = M^{1/2} w by the Lanczos process (Sec. IV.C), with the plan's mobility
// product as the operator.
//
// The Krylov basis V (one vector of dimension d = 3n, or 6n with torques, per iteration) stays on
// the device; every iteration runs one mobility product, two classical Gram-Schmidt passes against
// the whole basis (full re-orthogonalisation) and a norm, all as deterministic fixed-order
// reductions.  Three numbers per iteration (the two pass coefficients on the newest vector and the
// squared norm) go to the host, which builds the tridiagonal T_j, forms y_j = T_j^{1/2} e_1 from a
// Jacobi eigendecomposition and evaluates eps_j = ||y_j - [y_{j-1}; 0]|| / ||y_{j-1}||, which is
// ||g_j - g_{j-1}|| / ||g_{j-1}|| because the basis is orthonormal.  The result is
// g = ||w|| V_j y_j.
#include <math.h>
#include <string.h>

#include <algorithm>
#include <new>
#include <vector>

#include "dps_internal.cuh"

namespace dps {
namespace {

constexpr int kRedThreads = 256;
constexpr int kRedBlocks = 2 * 152;  // partial sums per reduction (fixed: the order never changes)
constexpr int kMaxLanczos = 128;

// part[k][b] = sum over the elements of block b's strided share of V_k . x, for k < nv
__global__ void __launch_bounds__(kRedThreads) dots_kernel(const double* __restrict__ V, int64_t ld, int nv,
                                                           const double* __restrict__ x, int64_t d,
                                                           double* __restrict__ part) {
  __shared__ double red[kRedThreads / 32];
  const int k = blockIdx.y;
  if (k >= nv) return;
  const double* v = V + (size_t)k * ld;
  double s = 0.0;
  for (int64_t i = (int64_t)blockIdx.x * kRedThreads + threadIdx.x; i < d; i += (int64_t)gridDim.x * kRedThreads)
    s = fma(v[i], x[i], s);
#pragma unroll
  for (int off = 16; off > 0; off >>= 1) s += __shfl_xor_sync(0xffffffffu, s, off);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = s;
  __syncthreads();
  if (threadIdx.x == 0) {
    double t = 0.0;
    for (int w = 0; w < kRedThreads / 32; ++w) t += red[w];
    part[(size_t)k * gridDim.x + blockIdx.x] = t;
  }
}

// out[k] = sum_b part[k][b] in a fixed order (one block per k)
__global__ void __launch_bounds__(kRedThreads) finish_kernel(const double* __restrict__ part, int nb,
                                                             double* __restrict__ out) {
  __shared__ double red[kRedThreads];
  const int k = blockIdx.x;
  double s = 0.0;
  for (int b = threadIdx.x; b < nb; b += kRedThreads) s += part[(size_t)k * nb + b];
  red[threadIdx.x] = s;
  __syncthreads();
  for (int h = kRedThreads / 2; h > 0; h >>= 1) {
    if ((int)threadIdx.x < h) red[threadIdx.x] += red[threadIdx.x + h];
    __syncthreads();
  }
  if (threadIdx.x == 0) out[k] = red[0];
}

// x[i] = a * x[i] + sum_{k < nv} c[k] V_k[i]   (c on the device, nv <= kMaxLanczos)
__global__ void __launch_bounds__(kRedThreads) combine_kernel(double* __restrict__ x, double a,
                                                              const double* __restrict__ V, int64_t ld, int nv,
                                                              const double* __restrict__ c, double cscale,
                                                              int64_t d) {
  __shared__ double sc[kMaxLanczos];
  for (int k = threadIdx.x; k < nv; k += kRedThreads) sc[k] = cscale * c[k];
  __syncthreads();
  for (int64_t i = (int64_t)blockIdx.x * kRedThreads + threadIdx.x; i < d; i += (int64_t)gridDim.x * kRedThreads) {
    double s = a == 0.0 ? 0.0 : a * x[i];
    for (int k = 0; k < nv; ++k) s = fma(sc[k], V[(size_t)k * ld + i], s);
    x[i] = s;
  }
}

// dst[i] = s * src[i]
__global__ void __launch_bounds__(kRedThreads) scale_kernel(double* __restrict__ dst, const double* __restrict__ src,
                                                            double s, int64_t d) {
  for (int64_t i = (int64_t)blockIdx.x * kRedThreads + threadIdx.x; i < d; i += (int64_t)gridDim.x * kRedThreads)
    dst[i] = s * src[i];
}

unsigned stream_blocks(int64_t d) {
  return (unsigned)std::max<int64_t>(1, std::min<int64_t>(4 * 152, (d + kRedThreads - 1) / kRedThreads));
}

// Eigendecomposition of a symmetric j x j matrix A (row-major, overwritten) by cyclic Jacobi
// rotations: after convergence A is diagonal (the eigenvalues) and Q (row-major) holds the
// eigenvectors as columns.  Each rotation zeroes one off-diagonal pair with the angle given by
// tau = (a_qq - a_pp) / (2 a_pq), t = sign(tau) / (|tau| + sqrt(1 + tau^2)).
void jacobi_eigen(int j, std::vector<double>& A, std::vector<double>& Q) {
  Q.assign((size_t)j * j, 0.0);
  for (int i = 0; i < j; ++i) Q[(size_t)i * j + i] = 1.0;
  double scale = 0.0;
  for (double v : A) scale = std::max(scale, fabs(v));
  if (scale == 0.0) return;
  for (int sweep = 0; sweep < 100; ++sweep) {
    double off = 0.0;
    for (int p = 0; p < j; ++p)
      for (int q = p + 1; q < j; ++q) off = std::max(off, fabs(A[(size_t)p * j + q]));
    if (off <= 1e-17 * scale) break;
    for (int p = 0; p < j; ++p) {
      for (int q = p + 1; q < j; ++q) {
        const double apq = A[(size_t)p * j + q];
        if (apq == 0.0) continue;
        const double tau = (A[(size_t)q * j + q] - A[(size_t)p * j + p]) / (2.0 * apq);
        const double t = (tau >= 0.0 ? 1.0 : -1.0) / (fabs(tau) + sqrt(1.0 + tau * tau));
        const double c = 1.0 / sqrt(1.0 + t * t), s = t * c;
        for (int k = 0; k < j; ++k) {  // columns p, q of A
          const double akp = A[(size_t)k * j + p], akq = A[(size_t)k * j + q];
          A[(size_t)k * j + p] = c * akp - s * akq;
          A[(size_t)k * j + q] = s * akp + c * akq;
        }
        for (int k = 0; k < j; ++k) {  // rows p, q of A
          const double apk = A[(size_t)p * j + k], aqk = A[(size_t)q * j + k];
          A[(size_t)p * j + k] = c * apk - s * aqk;
          A[(size_t)q * j + k] = s * apk + c * aqk;
        }
        for (int k = 0; k < j; ++k) {  // eigenvectors
          const double qkp = Q[(size_t)k * j + p], qkq = Q[(size_t)k * j + q];
          Q[(size_t)k * j + p] = c * qkp - s * qkq;
          Q[(size_t)k * j + q] = s * qkp + c * qkq;
        }
      }
    }
  }
}

}  // namespace

// y = T^{1/2} e_1 for the symmetric tridiagonal T (diagonal alpha[j], off-diagonal beta[j-1]);
// eigenvalues below zero take a zero square root
void tridiag_sqrt_e1(int j, const double* alpha, const double* beta, double* y) {
  std::vector<double> A((size_t)j * j, 0.0), Q;
  for (int i = 0; i < j; ++i) {
    A[(size_t)i * j + i] = alpha[i];
    if (i + 1 < j) A[(size_t)i * j + i + 1] = A[(size_t)(i + 1) * j + i] = beta[i];
  }
  jacobi_eigen(j, A, Q);
  for (int r = 0; r < j; ++r) y[r] = 0.0;
  for (int i = 0; i < j; ++i) {
    const double s = sqrt(std::max(A[(size_t)i * j + i], 0.0)) * Q[i];  // Q[0][i]
    for (int r = 0; r < j; ++r) y[r] += Q[(size_t)r * j + i] * s;
  }
}

struct Lanczos {
  Plan* plan;
  int max_iter;
  int64_t dmax;   // vector dimension at max_n
  double* V;      // [max_iter][dmax] basis
  double* R;      // [dmax] work vector (the next basis vector before normalisation)
  double* part;   // [max_iter][kRedBlocks] partial sums
  double* coef;   // [2][max_iter] Gram-Schmidt coefficients of the two passes, then [1] squared norm
  double* y;      // [max_iter] host-built combination coefficients
  double* h_out;  // pinned host copy of the three numbers per iteration
};

}  // namespace dps

using dps::Lanczos;

extern "C" {

dps_status dpstokes_tridiag_sqrt_e1(int32_t j, const double* alpha, const double* beta, double* y) {
  if (j < 1 || j > dps::kMaxLanczos || !alpha || !y || (j > 1 && !beta)) return DPS_ERR_INVALID_ARG;
  dps::tridiag_sqrt_e1(j, alpha, beta, y);
  return DPS_OK;
}

dps_status dpstokes_lanczos_create(dps_lanczos_t* out, dps_plan_t plan, int32_t max_iter) {
  if (!out) return DPS_ERR_INVALID_ARG;
  *out = nullptr;
  dps::Plan* p = reinterpret_cast<dps::Plan*>(plan);
  if (!p || max_iter < 2 || max_iter > dps::kMaxLanczos) return DPS_ERR_INVALID_ARG;
  Lanczos* lz = new (std::nothrow) Lanczos();
  if (!lz) return DPS_ERR_OOM;
  memset(lz, 0, sizeof(Lanczos));
  lz->plan = p;
  lz->max_iter = max_iter;
  lz->dmax = (p->g.with_torque ? 6 : 3) * std::max<int64_t>(p->max_n, 1);
  int dev = -1;
  cudaGetDevice(&dev);
  if (dev != p->device) cudaSetDevice(p->device);
  const size_t vb = (size_t)lz->dmax * sizeof(double);
  bool ok = cudaMalloc(&lz->V, vb * max_iter) == cudaSuccess && cudaMalloc(&lz->R, vb) == cudaSuccess &&
            cudaMalloc(&lz->part, sizeof(double) * dps::kRedBlocks * max_iter) == cudaSuccess &&
            cudaMalloc(&lz->coef, sizeof(double) * (2 * max_iter + 1)) == cudaSuccess &&
            cudaMalloc(&lz->y, sizeof(double) * max_iter) == cudaSuccess &&
            cudaMallocHost(&lz->h_out, sizeof(double) * (2 * max_iter + 1)) == cudaSuccess;
  if (dev != p->device && dev >= 0) cudaSetDevice(dev);
  if (!ok) {
    cudaGetLastError();
    dpstokes_lanczos_destroy(reinterpret_cast<dps_lanczos_t>(lz));
    return DPS_ERR_OOM;
  }
  *out = reinterpret_cast<dps_lanczos_t>(lz);
  return DPS_OK;
}

void dpstokes_lanczos_destroy(dps_lanczos_t handle) {
  Lanczos* lz = reinterpret_cast<Lanczos*>(handle);
  if (!lz) return;
  cudaDeviceSynchronize();
  if (lz->V) cudaFree(lz->V);
  if (lz->R) cudaFree(lz->R);
  if (lz->part) cudaFree(lz->part);
  if (lz->coef) cudaFree(lz->coef);
  if (lz->y) cudaFree(lz->y);
  if (lz->h_out) cudaFreeHost(lz->h_out);
  delete lz;
}

dps_status dpstokes_lanczos_sample(dps_lanczos_t handle, int64_t n, const double* positions, const double* w,
                                   double* g, double tol, int32_t* iters, double* eps, double* eps_hist,
                                   void* stream) {
  using namespace dps;
  Lanczos* lz = reinterpret_cast<Lanczos*>(handle);
  if (!lz) return DPS_ERR_INVALID_ARG;
  Plan* p = lz->plan;
  if (n < 0 || n > p->max_n || !(tol >= 0.0)) return DPS_ERR_INVALID_ARG;
  if (n > 0 && (!positions || !w || !g)) return DPS_ERR_INVALID_ARG;
  if (iters) *iters = 0;
  if (eps) *eps = 0.0;
  if (n == 0) return DPS_OK;
  cudaStream_t s = (cudaStream_t)stream;
  const bool tq = p->g.with_torque != 0;
  const int64_t d = (tq ? 6 : 3) * n, ld = lz->dmax;
  const unsigned sb = stream_blocks(d);
  int dev = -1;
  cudaGetDevice(&dev);
  if (dev != p->device) cudaSetDevice(p->device);
  dps_status st = DPS_OK;
  auto fail = [&](dps_status e) {
    if (dev != p->device && dev >= 0) cudaSetDevice(dev);
    return e;
  };
  // squared norm of x into coef[slot] and the host copy
  auto norm2 = [&](const double* x, int slot) {
    dots_kernel<<<dim3(kRedBlocks, 1), kRedThreads, 0, s>>>(x, 0, 1, x, d, lz->part);
    finish_kernel<<<1, kRedThreads, 0, s>>>(lz->part, kRedBlocks, lz->coef + slot);
  };
  norm2(w, 2 * lz->max_iter);
  if (cudaMemcpyAsync(lz->h_out, lz->coef + 2 * lz->max_iter, sizeof(double), cudaMemcpyDeviceToHost, s) !=
          cudaSuccess ||
      cudaStreamSynchronize(s) != cudaSuccess)
    return fail(DPS_ERR_CUDA);
  const double beta0 = sqrt(lz->h_out[0]);
  if (!isfinite(beta0)) return fail(DPS_ERR_NONFINITE);
  if (beta0 == 0.0) {
    if (cudaMemsetAsync(g, 0, sizeof(double) * d, s) != cudaSuccess) return fail(DPS_ERR_CUDA);
    return fail(dpstokes_status(reinterpret_cast<dps_plan_t>(p), stream));
  }
  scale_kernel<<<sb, kRedThreads, 0, s>>>(lz->V, w, 1.0 / beta0, d);
  std::vector<double> alpha, beta, y, yprev;
  int j = 0;
  double last_eps = 0.0;
  for (j = 1; j <= lz->max_iter; ++j) {
    double* vj = lz->V + (size_t)(j - 1) * ld;
    // R = M v_j
    st = run(p, n, positions, vj, tq ? vj + 3 * n : nullptr, lz->R, tq ? lz->R + 3 * n : nullptr, s, 99);
    if (st != DPS_OK) return fail(st);
    // two Gram-Schmidt passes against v_1..v_j, then |R|^2
    for (int pass = 0; pass < 2; ++pass) {
      double* c = lz->coef + pass * lz->max_iter;
      dots_kernel<<<dim3(kRedBlocks, j), kRedThreads, 0, s>>>(lz->V, ld, j, lz->R, d, lz->part);
      finish_kernel<<<j, kRedThreads, 0, s>>>(lz->part, kRedBlocks, c);
      combine_kernel<<<sb, kRedThreads, 0, s>>>(lz->R, 1.0, lz->V, ld, j, c, -1.0, d);
    }
    norm2(lz->R, 2 * lz->max_iter);
    // the coefficients on v_j of both passes and the norm
    if (cudaMemcpyAsync(lz->h_out, lz->coef + (j - 1), sizeof(double), cudaMemcpyDeviceToHost, s) != cudaSuccess ||
        cudaMemcpyAsync(lz->h_out + 1, lz->coef + lz->max_iter + (j - 1), sizeof(double), cudaMemcpyDeviceToHost,
                        s) != cudaSuccess ||
        cudaMemcpyAsync(lz->h_out + 2, lz->coef + 2 * lz->max_iter, sizeof(double), cudaMemcpyDeviceToHost, s) !=
            cudaSuccess ||
        cudaStreamSynchronize(s) != cudaSuccess)
      return fail(DPS_ERR_CUDA);
    if (cudaGetLastError() != cudaSuccess) return fail(DPS_ERR_CUDA);
    const double a = lz->h_out[0] + lz->h_out[1], b = sqrt(std::max(lz->h_out[2], 0.0));
    if (!isfinite(a) || !isfinite(b)) {
      st = dpstokes_status(reinterpret_cast<dps_plan_t>(p), stream);
      return fail(st != DPS_OK ? st : DPS_ERR_NONFINITE);
    }
    alpha.push_back(a);
    y.assign(j, 0.0);
    tridiag_sqrt_e1(j, alpha.data(), beta.data(), y.data());
    bool done = (b == 0.0) || j == lz->max_iter;
    if (j >= 2) {
      double dn = 0.0, pn = 0.0;
      for (int r = 0; r < j; ++r) {
        const double pr = r < j - 1 ? yprev[r] : 0.0;
        dn += (y[r] - pr) * (y[r] - pr);
        pn += pr * pr;
      }
      last_eps = sqrt(dn) / sqrt(pn);
      if (eps_hist) eps_hist[j - 2] = last_eps;
      if (last_eps <= tol) done = true;
    }
    yprev = y;
    if (done) break;
    beta.push_back(b);
    scale_kernel<<<sb, kRedThreads, 0, s>>>(lz->V + (size_t)j * ld, lz->R, 1.0 / b, d);
  }
  if (j > lz->max_iter) j = lz->max_iter;
  // g = beta_0 V_j y_j
  if (cudaMemcpyAsync(lz->y, y.data(), sizeof(double) * j, cudaMemcpyHostToDevice, s) != cudaSuccess)
    return fail(DPS_ERR_CUDA);
  combine_kernel<<<sb, kRedThreads, 0, s>>>(g, 0.0, lz->V, ld, j, lz->y, beta0, d);
  if (cudaGetLastError() != cudaSuccess) return fail(DPS_ERR_CUDA);
  if (iters) *iters = j;
  if (eps) *eps = last_eps;
  st = dpstokes_status(reinterpret_cast<dps_plan_t>(p), stream);  // synchronises; reads the device checks
  return fail(st);
}

}  // extern "C"
