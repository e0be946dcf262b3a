// Stochastic drift by random finite differences (Sec. IV.C, footnote on Brownian dynamics in
// confinement): d = (1/delta) [M(q + delta/2 W) - M(q - delta/2 W)] [W; 0], whose average over a
// standard normal W is the divergence of the mobility with respect to the positions q.  Two products
// of the plan; the displaced positions and the first product live in the plan's staging buffers.
// Stream-ordered, no host synchronisation, no allocation.
#include "dps_internal.cuh"

namespace dps {
namespace {

// qp = q + (delta/2) W, qm = q - (delta/2) W; zero torques when the plan takes torques
__global__ void displace_kernel(int64_t n3, const double* __restrict__ q, const double* __restrict__ W, double hd,
                                double* __restrict__ qp, double* __restrict__ qm, double* __restrict__ t0) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n3) return;
  const double s = hd * W[i];
  qp[i] = q[i] + s;
  qm[i] = q[i] - s;
  if (t0) t0[i] = 0.0;
}

// out = (a - out) / delta
__global__ void difference_kernel(int64_t m, const double* __restrict__ a, double inv_delta, double* __restrict__ out) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= m) return;
  out[i] = (a[i] - out[i]) * inv_delta;
}

}  // namespace
}  // namespace dps

extern "C" dps_status dpstokes_rfd_drift(dps_plan_t plan, int64_t n, const double* positions, const double* W,
                                         double delta, double* out, void* stream) {
  using namespace dps;
  Plan* p = reinterpret_cast<Plan*>(plan);
  if (!p || n < 0 || n > p->max_n || !(delta > 0.0) || !isfinite(delta)) return DPS_ERR_INVALID_ARG;
  if (n > 0 && (!positions || !W || !out)) return DPS_ERR_INVALID_ARG;
  if (n == 0) return DPS_OK;
  cudaStream_t s = (cudaStream_t)stream;
  const bool tq = p->g.with_torque != 0;
  const size_t m = (size_t)p->max_n;
  // staging: [q+ | q- | zero torques] in stage_in (9 max_n doubles), the first product in stage_out
  double* qp = p->stage_in;
  double* qm = qp + 3 * m;
  double* t0 = tq ? qm + 3 * m : nullptr;
  double* U1 = p->stage_out;
  double* W1 = tq ? U1 + 3 * m : nullptr;
  int dev = -1;
  cudaGetDevice(&dev);
  if (dev != p->device) cudaSetDevice(p->device);
  const int64_t n3 = 3 * n;
  const int threads = 256;
  displace_kernel<<<(unsigned)((n3 + threads - 1) / threads), threads, 0, s>>>(n3, positions, W, 0.5 * delta, qp, qm,
                                                                               t0);
  dps_status st = run(p, n, qp, W, t0, U1, W1, s, 99);
  if (st == DPS_OK) st = run(p, n, qm, W, t0, out, tq ? out + 3 * n : nullptr, s, 99);
  if (st == DPS_OK) {
    difference_kernel<<<(unsigned)((n3 + threads - 1) / threads), threads, 0, s>>>(n3, U1, 1.0 / delta, out);
    if (tq)
      difference_kernel<<<(unsigned)((n3 + threads - 1) / threads), threads, 0, s>>>(n3, W1, 1.0 / delta, out + 3 * n);
    if (cudaGetLastError() != cudaSuccess) st = DPS_ERR_CUDA;
  }
  if (dev != p->device && dev >= 0) cudaSetDevice(dev);
  return st;
}
