// Particle-side kernels: envelope records, binning, spreading (step 1 of Sec. III.D) and
// interpolation (step 8, Eqs. 10-11) of the doubly-periodic FCM mobility product.
//
// Envelope: Delta^W(x - r_j) = phi(dx) phi(dy) [phi(dz) - s_b phi(z - z_im,bottom)
//                                                      - s_t phi(z - z_im,top)]   (Eqs. 9, 53, 54)
// phi(t) = exp(beta (sqrt(1 - (t/alpha)^2) - 1)) / Z on |t| <= alpha, zero outside.
//
// Each particle gets one record per apply holding its force/torque and the separable envelope
// factors at the nodes of its support (x and y slots, and the Chebyshev nodes of its z support
// with the wall images folded in).  Spreading and interpolation both read these records, so the
// two operators use bit-identical weights (they are adjoint under the quadrature).
//
// Spreading is a gather: one block owns a 32 x 8 tile of xy nodes over all occupied Chebyshev
// planes, collects the particles whose support touches the tile from the surrounding bins, and
// writes every node of its tile exactly once with plain stores (no atomics, no zero-fill pass).
// Interpolation is a warp per particle: lane groups walk the x run of each (z, y) row of the
// support, so every row is read as one contiguous segment.
//
// Torques take one of the two routes of Sec. III.D.  Spectral curl: the torque envelopes are spread
// as three more fields (the half-curl is formed in Fourier-Chebyshev space).  Kernel derivative:
// the records also hold the truncated derivative phi' of the dipole kernel in x, y and (imaged) z,
// the spread adds (1/2) grad Delta_D x tau to the force density, and interpolation returns
// Omega_j = (1/2) h^2 sum_g w_c u(x_g) x grad Delta_D(x_g - r_j).
#include <cuda.h>
#include <cudaTypedefs.h>
#include <limits.h>
#include <math.h>

#include <algorithm>
#include <type_traits>

#include "dps_internal.cuh"

namespace dps {

namespace {

__device__ __forceinline__ double es_eval(double t, const EsKernel& k) {
  const double r = t / k.alpha;
  if (fabs(r) > 1.0) return 0.0;
  return exp(k.beta * (sqrt(1.0 - r * r) - 1.0)) * k.inv_norm;
}

__device__ __forceinline__ float es_eval_f(double t, const EsKernel& k) {
  // the offset t is formed in double by the caller (a difference of nearby large numbers); the
  // rest runs in float, narrowed on the integer pipe toward zero (a division or a conversion in
  // double occupies the scarce FP64 pipe; toward zero, a node inside the support stays inside)
  const float r = narrow_bits(t) * k.inv_alpha_f;
  if (fabsf(r) > 1.0f) return 0.0f;
  const float q = fmaxf(0.0f, 1.0f - r * r);
  return expf(k.beta_f * (sqrtf(q) - 1.0f)) * k.inv_norm_f;
}

template <typename T> __device__ __forceinline__ T es_t(double t, const EsKernel& k);
template <> __device__ __forceinline__ double es_t<double>(double t, const EsKernel& k) { return es_eval(t, k); }
template <> __device__ __forceinline__ float es_t<float>(double t, const EsKernel& k) { return es_eval_f(t, k); }

// derivative of the ES kernel, phi'(t) = -beta t / (alpha^2 sqrt(1 - (t/alpha)^2)) phi(t), zero for
// |t| > cut (the point where |phi'| is smallest before it blows up at the support edge)
__device__ __forceinline__ double esd_eval(double t, const EsKernel& k) {
  if (fabs(t) > k.cut) return 0.0;
  const double r = t / k.alpha;
  const double s = sqrt(1.0 - r * r);
  return -k.beta * r / (k.alpha * s) * exp(k.beta * (s - 1.0)) * k.inv_norm;
}

__device__ __forceinline__ float esd_eval_f(double t, const EsKernel& k) {
  // the truncation is decided in double, as on the double path: a node cut on one side and kept on
  // the other would change a result by |phi'(cut)|, far above float rounding.  The bit patterns of
  // non-negative doubles order as the values, so the test runs on the integer pipe.
  if ((__double_as_longlong(t) & 0x7fffffffffffffffLL) > __double_as_longlong(k.cut)) return 0.0f;
  const float r = narrow_bits(t) * k.inv_alpha_f;
  const float s = sqrtf(fmaxf(0.0f, 1.0f - r * r));
  return -k.beta_over_alpha_f * r / s * expf(k.beta_f * (s - 1.0f)) * k.inv_norm_f;
}

template <typename T> __device__ __forceinline__ T esd_t(double t, const EsKernel& k);
template <> __device__ __forceinline__ double esd_t<double>(double t, const EsKernel& k) { return esd_eval(t, k); }
template <> __device__ __forceinline__ float esd_t<float>(double t, const EsKernel& k) { return esd_eval_f(t, k); }

__device__ __forceinline__ int wrap_idx(int i, int n) {
  i %= n;
  return i < 0 ? i + n : i;
}

// first node index a with |a h - x| <= alpha (candidates start at floor((x - alpha)/h))
__device__ __forceinline__ int first_node(double x, double h, double inv_h, double alpha) {
  int a = (int)floor((x - alpha) * inv_h);
  if (fabs((double)a * h - x) > alpha) ++a;
  return a;
}

// number of Chebyshev nodes with z_c > v (nodes decrease with c)
__device__ __forceinline__ int count_above(const double* zc, int nz, double v) {
  int lo = 0, hi = nz;  // answer in [0, nz]
  while (lo < hi) {
    const int mid = (lo + hi) >> 1;
    if (zc[mid] > v) lo = mid + 1; else hi = mid;
  }
  return lo;
}

// One thread per particle.  STAGED: the block's records are built in shared memory and then
// copied to their contiguous place in global memory with 16-byte stores (a thread writing its own
// record directly would make every warp store touch 32 different sectors).
template <typename T, bool STAGED>
__global__ void records_kernel(Geometry g, int64_t n, const double* __restrict__ pos,
                               const double* __restrict__ F, const double* __restrict__ Tq,
                               const double* __restrict__ zc, uint32_t* __restrict__ rec,
                               int* __restrict__ bin_of, int* __restrict__ bin_count,
                               int* __restrict__ zrange, int* __restrict__ status) {
  extern __shared__ __align__(16) uint32_t srec_out[];
  const int64_t j0 = (int64_t)blockIdx.x * blockDim.x;
  const int64_t j = j0 + threadIdx.x;
  if (!STAGED && j >= n) return;
  if (j < n) {
  uint32_t* r = STAGED ? srec_out + (size_t)threadIdx.x * g.rec_words : rec + (size_t)j * g.rec_words;
  T* tv = reinterpret_cast<T*>(r + 8);
  double x = pos[3 * j], y = pos[3 * j + 1], z = pos[3 * j + 2];
  double f[3] = {F[3 * j], F[3 * j + 1], F[3 * j + 2]};
  double tq[3] = {0.0, 0.0, 0.0};
  if (g.with_torque) { tq[0] = Tq[3 * j]; tq[1] = Tq[3 * j + 1]; tq[2] = Tq[3 * j + 2]; }
  bool finite = isfinite(x) && isfinite(y) && isfinite(z);
  for (int i = 0; i < 3; ++i) finite = finite && isfinite(f[i]) && isfinite(tq[i]);
  bool ok = finite;
  if (!finite) atomicOr(status, kStatNonfinite);
  double amax = g.kM.alpha;
  if (g.with_torque && g.kD.alpha > amax) amax = g.kD.alpha;
  if (ok) {
    bool in_dom = (z >= g.zmin) && (z <= g.zmax);
    if (g.mode == DPS_FREE && z - amax < g.zmin) in_dom = false;
    if ((g.mode == DPS_FREE || g.mode == DPS_BOTTOM_WALL) && z + amax > g.zmax) in_dom = false;
    if (!in_dom) { atomicOr(status, kStatDomain); ok = false; }
  }
  // wrap x, y into [0, L)
  double xw = 0.0, yw = 0.0;
  if (ok) {
    xw = x - g.Lx * floor(x / g.Lx);
    if (xw >= g.Lx) xw -= g.Lx;
    if (xw < 0.0) xw = 0.0;
    yw = y - g.Ly * floor(y / g.Ly);
    if (yw >= g.Ly) yw -= g.Ly;
    if (yw < 0.0) yw = 0.0;
  }
  const double tscale = g.torque_deriv ? 0.5 : 1.0;  // the derivative route stores tau / 2
  for (int i = 0; i < 3; ++i) {
    tv[i] = ok ? (T)f[i] : (T)0;
    tv[3 + i] = ok ? (T)(tscale * tq[i]) : (T)0;
  }
  int cmin = g.nz, cmax = -1;
  const int stride = 2 * g.pxc + g.lzc;
  for (int K = 0; K < g.nkernels; ++K) {
    const EsKernel& k = (K == 0) ? g.kM : g.kD;
    int4 hd = make_int4(0, 0, 0, 0);
    T* ph = tv + 6 + K * stride;
    if (ok) {
      const int ax = first_node(xw, g.h, g.inv_h, k.alpha);
      const int ay = first_node(yw, g.h, g.inv_h, k.alpha);
      const double tx0 = (double)ax * g.h - xw, ty0 = (double)ay * g.h - yw;  // offsets of the first nodes
      {
        double tx = tx0, ty = ty0;  // node offsets by running sums (one add each per slot)
        for (int i = 0; i < g.pxc; ++i) {
          ph[i] = (i < k.px) ? es_t<T>(tx, k) : (T)0;
          ph[g.pxc + i] = (i < k.px) ? es_t<T>(ty, k) : (T)0;
          tx += g.h;
          ty += g.h;
        }
      }
      hd.x = wrap_idx(ax, g.nx);
      hd.y = wrap_idx(ay, g.ny);
      // z support: nodes with z_c in [max(zmin, z - alpha), min(zmax, z + alpha)], widened by a
      // hair so that the exact |t| <= alpha tests below decide membership
      const double eps = 1e-12 * (g.H + fabs(z));
      const int c0 = count_above(zc, g.nz, z + k.alpha + eps);
      const int c1 = count_above(zc, g.nz, z - k.alpha - eps) - 1;
      int cnt = c1 - c0 + 1;
      if (cnt < 0) cnt = 0;
      if (cnt > g.lzc) { cnt = g.lzc; atomicOr(status, kStatInternal); }
      hd.z = c0;
      hd.w = cnt;
      const bool bottom_img = (g.mode == DPS_BOTTOM_WALL || g.mode == DPS_SLIT);
      const bool top_img = (g.mode == DPS_SLIT);
      for (int i = 0; i < g.lzc; ++i) {
        T v = (T)0;
        if (i < cnt) {
          const double zz = zc[c0 + i];
          T acc = es_t<T>(zz - z, k);
          if (bottom_img) acc -= es_t<T>(zz - (2.0 * g.zmin - z), k);
          if (top_img) acc -= es_t<T>(zz - (2.0 * g.zmax - z), k);
          v = acc;
        }
        ph[2 * g.pxc + i] = v;
      }
      if (K == 1 && g.torque_deriv) {
        // derivative slab: phi' in x and y, and d/dz of the imaged z factor (the exact derivative
        // of the negatively imaged envelope)
        T* pd = tv + 6 + 2 * stride;
        double tx = tx0, ty = ty0;
        for (int i = 0; i < g.pxc; ++i) {
          pd[i] = (i < k.px) ? esd_t<T>(tx, k) : (T)0;
          pd[g.pxc + i] = (i < k.px) ? esd_t<T>(ty, k) : (T)0;
          tx += g.h;
          ty += g.h;
        }
        for (int i = 0; i < g.lzc; ++i) {
          T v = (T)0;
          if (i < cnt) {
            const double zz = zc[c0 + i];
            T acc = esd_t<T>(zz - z, k);
            if (bottom_img) acc -= esd_t<T>(zz - (2.0 * g.zmin - z), k);
            if (top_img) acc -= esd_t<T>(zz - (2.0 * g.zmax - z), k);
            v = acc;
          }
          pd[2 * g.pxc + i] = v;
        }
      }
      if (cnt > 0) {
        cmin = min(cmin, c0);
        cmax = max(cmax, c0 + cnt - 1);
      }
    } else {
      const int nv = (K == 1 && g.torque_deriv) ? 2 * stride : stride;  // slab K (and the derivatives)
      for (int i = 0; i < nv; ++i) ph[i] = (T)0;
    }
    reinterpret_cast<int4*>(r)[K] = hd;
  }
  if (g.nkernels == 1) reinterpret_cast<int4*>(r)[1] = make_int4(0, 0, 0, 0);
  int bx = 0, by = 0;
  if (ok) {
    bx = min((int)floor(xw * g.inv_h) / kTileX, g.nbx - 1);
    by = min((int)floor(yw * g.inv_h) / kTileY, g.nby - 1);
  }
  const int b = by * g.nbx + bx;
  bin_of[j] = b;
  atomicAdd(&bin_count[b], 1);
  if (cmax >= 0) {
    atomicMin(&zrange[0], cmin);
    atomicMax(&zrange[1], cmax);
  }
  }  // j < n
  if (STAGED) {
    __syncthreads();
    const int64_t left = n - j0;
    const int cnt = left < (int64_t)blockDim.x ? (int)left : (int)blockDim.x;
    const int q = cnt * (g.rec_words / 4);  // 16-byte pieces (rec_words is a multiple of 4)
    const uint4* src = reinterpret_cast<const uint4*>(srec_out);
    uint4* dst = reinterpret_cast<uint4*>(rec + (size_t)j0 * g.rec_words);
    for (int t = threadIdx.x; t < q; t += blockDim.x) dst[t] = src[t];
  }
}

// exclusive scan of bin counts (one block; bins handled in contiguous chunks per thread)
__global__ void bin_scan_kernel(const int* __restrict__ count, int* __restrict__ start,
                                int* __restrict__ cursor, int nbins) {
  __shared__ int part[1024];
  const int t = threadIdx.x;
  const int per = (nbins + blockDim.x - 1) / blockDim.x;
  const int b0 = t * per, b1 = min(nbins, b0 + per);
  int s = 0;
  for (int b = b0; b < b1; ++b) s += count[b];
  part[t] = s;
  __syncthreads();
  for (int off = 1; off < (int)blockDim.x; off <<= 1) {
    const int v = (t >= off) ? part[t - off] : 0;
    __syncthreads();
    part[t] += v;
    __syncthreads();
  }
  int run = part[t] - s;
  for (int b = b0; b < b1; ++b) {
    start[b] = run;
    cursor[b] = run;
    run += count[b];
  }
  if (t == blockDim.x - 1) start[nbins] = part[t];
}

__global__ void bin_scatter_kernel(int64_t n, const int* __restrict__ bin_of, int* __restrict__ cursor,
                                   int* __restrict__ sorted) {
  const int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (j >= n) return;
  const int p = atomicAdd(&cursor[bin_of[j]], 1);
  sorted[p] = (int)j;
}

// Particles of one bin in increasing index order (the scatter's atomics leave the order open), so
// the spread sums in the same order on every apply: results repeat bit for bit.  One thread per bin,
// insertion sort; bins above kSortedBinMax particles keep the scatter's order.
constexpr int kSortedBinMax = 256;

__global__ void bin_sort_kernel(const int* __restrict__ start, int* __restrict__ sorted, int nbins) {
  const int b = blockIdx.x * blockDim.x + threadIdx.x;
  if (b >= nbins) return;
  const int s0 = start[b], s1 = start[b + 1];
  if (s1 - s0 < 2 || s1 - s0 > kSortedBinMax) return;
  for (int i = s0 + 1; i < s1; ++i) {
    const int v = sorted[i];
    int j = i - 1;
    while (j >= s0 && sorted[j] > v) {
      sorted[j + 1] = sorted[j];
      --j;
    }
    sorted[j + 1] = v;
  }
}

// does the cyclic node interval [a, a+len_a) intersect [b, b+len_b) (mod n)?
__device__ __forceinline__ bool cyc_overlap(int a, int len_a, int b, int len_b, int n) {
  int d1 = b - a; if (d1 < 0) d1 += n;
  int d2 = a - b; if (d2 < 0) d2 += n;
  return d1 < len_a || d2 < len_b;
}

constexpr int kCandCap = 2048;
constexpr int kStage = 128;  // candidate records staged in shared memory at a time

// Candidate e of a list: a warp-wide row list (int staged indices) or, with LANE, this lane's own
// list of byte indices stored [e][32 lanes].
template <bool LANE>
__device__ __forceinline__ int list_entry(const void* wl, int e) {
  if (LANE) return (int)static_cast<const unsigned char*>(wl)[e * 32 + (threadIdx.x & 31)];
  return static_cast<const int*>(wl)[e];
}

constexpr int kLaneCap = 32;  // entries of a per-lane candidate list

// Per lane (node column gx) of a warp, the candidates of the warp's row list whose x support covers
// gx (record head K), as byte indices into the staged records; returns the count, which may exceed
// kLaneCap (the caller then keeps the row list).  A candidate covers about 6 of the 32 columns, so
// the walks over the z chunks visit about a fifth of the row list per lane.
template <int K>
__device__ __forceinline__ int build_lane_list(const Geometry& g, const uint32_t* srec, const int* wl, int nl, int rw,
                                               int gx, bool active, unsigned char* ll) {
  const int lane = threadIdx.x & 31;
  const int px = (K == 0) ? g.kM.px : g.kD.px;
  int cnt = 0;
  for (int e = 0; e < nl; ++e) {
    const int idx = wl[e];
    const int4 hd = reinterpret_cast<const int4*>(srec + (size_t)idx * rw)[K];
    int dx = gx - hd.x;
    if (dx < 0) dx += g.nx;
    if (active && dx < px) {
      if (cnt < kLaneCap) ll[cnt * 32 + lane] = (unsigned char)idx;
      ++cnt;
    }
  }
  return cnt;
}

// Per warp (one tile row gy), the staged candidates whose support rows include gy, one list per
// kernel (monopole / dipole, the latter when TWO), built with warp ballots; the z-chunk loops then
// walk only these.
template <bool TWO>
__device__ __forceinline__ void build_row_lists(const Geometry& g, const uint32_t* srec, int nrec, int rw, int gy,
                                                int* wl0, int* wl1, int& n0, int& n1) {
  const int lane = threadIdx.x & 31;
  n0 = n1 = 0;
  for (int base = 0; base < nrec; base += 32) {
    const int i = base + lane;
    bool h0 = false, h1 = false;
    if (i < nrec) {
      const int4* hd = reinterpret_cast<const int4*>(srec + (size_t)i * rw);
      const int4 a = hd[0];
      int dy = gy - a.y;
      if (dy < 0) dy += g.ny;
      h0 = a.w > 0 && dy < g.kM.px;
      if (TWO) {
        const int4 b = hd[1];
        int dy1 = gy - b.y;
        if (dy1 < 0) dy1 += g.ny;
        h1 = b.w > 0 && dy1 < g.kD.px;
      }
    }
    const unsigned below = (1u << lane) - 1u;
    const unsigned m0 = __ballot_sync(0xffffffffu, h0);
    if (h0) wl0[n0 + __popc(m0 & below)] = i;
    n0 += __popc(m0);
    if (TWO) {
      const unsigned m1 = __ballot_sync(0xffffffffu, h1);
      if (h1) wl1[n1 + __popc(m1 & below)] = i;
      n1 += __popc(m1);
    }
  }
  __syncwarp();
}

// Accumulate the listed candidates of kernel K into the thread's node column (the three fields of
// that kernel), planes [zb, zb + ZC).
template <typename T, int ZC, int K, bool LANE>
__device__ __forceinline__ void spread_list(const Geometry& g, const uint32_t* srec, const void* wl, int nl, int rw,
                                            int gx, int gy, int zb, T (&acc)[ZC][3]) {
  const int stride = 2 * g.pxc + g.lzc;
  const int px = (K == 0) ? g.kM.px : g.kD.px;
  for (int e = 0; e < nl; ++e) {
    const uint32_t* r = srec + (size_t)list_entry<LANE>(wl, e) * rw;
    const int4 hd = reinterpret_cast<const int4*>(r)[K];
    if (hd.z + hd.w <= zb || hd.z >= zb + ZC) continue;  // no plane of this chunk (uniform)
    int dx = gx - hd.x;
    if (dx < 0) dx += g.nx;
    if (!LANE && dx >= px) continue;  // a lane list holds only candidates that cover gx
    int dy = gy - hd.y;
    if (dy < 0) dy += g.ny;
    const T* tv = reinterpret_cast<const T*>(r + 8);
    const T* ph = tv + 6 + K * stride;
    const T wxy = ph[dx] * ph[g.pxc + dy];
    const T f0 = tv[3 * K], f1 = tv[3 * K + 1], f2 = tv[3 * K + 2];
#pragma unroll
    for (int zz = 0; zz < ZC; ++zz) {
      const int iz = zb + zz - hd.z;
      if (iz >= 0 && iz < hd.w) {
        const T w = wxy * ph[2 * g.pxc + iz];
        acc[zz][0] += f0 * w;
        acc[zz][1] += f1 * w;
        acc[zz][2] += f2 * w;
      }
    }
  }
}

// Kernel-derivative torque route: accumulate the listed candidates' half-curl sources
// (1/2) grad Delta_D x tau into the thread's node column (the three force-density fields), planes
// [zb, zb + ZC).  The records hold tau / 2.  With gx = phi'x phiy phiz, gy = phix phi'y phiz and
// gz = phix phiy phi'z, grad Delta x tau = (gy tz - gz ty, gz tx - gx tz, gx ty - gy tx).
template <typename T, int ZC, bool LANE>
__device__ __forceinline__ void spread_curl_list(const Geometry& g, const uint32_t* srec, const void* wl, int nl,
                                                 int rw, int gx, int gy, int zb, T (&acc)[ZC][3]) {
  const int stride = 2 * g.pxc + g.lzc;
  const int px = g.kD.px;
  for (int e = 0; e < nl; ++e) {
    const uint32_t* r = srec + (size_t)list_entry<LANE>(wl, e) * rw;
    const int4 hd = reinterpret_cast<const int4*>(r)[1];
    if (hd.z + hd.w <= zb || hd.z >= zb + ZC) continue;  // no plane of this chunk (uniform)
    int dx = gx - hd.x;
    if (dx < 0) dx += g.nx;
    if (!LANE && dx >= px) continue;  // a lane list holds only candidates that cover gx
    int dy = gy - hd.y;
    if (dy < 0) dy += g.ny;
    const T* tv = reinterpret_cast<const T*>(r + 8);
    const T* ph = tv + 6 + stride;      // dipole phi
    const T* pd = tv + 6 + 2 * stride;  // dipole phi'
    const T fx = ph[dx], fy = ph[g.pxc + dy];
    const T wxy = fx * fy, bx = pd[dx] * fy, by = fx * pd[g.pxc + dy];
    const T tx = tv[3], ty = tv[4], tz = tv[5];
    const T a0 = by * tz, b0 = -wxy * ty;    // field 0: a0 phiz + b0 phi'z
    const T a1 = -bx * tz, b1 = wxy * tx;    // field 1: a1 phiz + b1 phi'z
    const T a2 = bx * ty - by * tx;          // field 2: a2 phiz
#pragma unroll
    for (int zz = 0; zz < ZC; ++zz) {
      const int iz = zb + zz - hd.z;
      if (iz >= 0 && iz < hd.w) {
        const T pz = ph[2 * g.pxc + iz], dz = pd[2 * g.pxc + iz];
        acc[zz][0] += a0 * pz + b0 * dz;
        acc[zz][1] += a1 * pz + b1 * dz;
        acc[zz][2] += a2 * pz;
      }
    }
  }
}

// Kernel-derivative route with coinciding supports (m_M = m_D, so both record heads are equal): each
// listed candidate adds F Delta_M and (1/2) grad Delta_D x tau in one walk.
template <typename T, int ZC, bool LANE>
__device__ __forceinline__ void spread_fused_list(const Geometry& g, const uint32_t* srec, const void* wl, int nl,
                                                  int rw, int gx, int gy, int zb, T (&acc)[ZC][3]) {
  const int stride = 2 * g.pxc + g.lzc;
  const int px = g.kM.px;
  for (int e = 0; e < nl; ++e) {
    const uint32_t* r = srec + (size_t)list_entry<LANE>(wl, e) * rw;
    const int4 hd = reinterpret_cast<const int4*>(r)[0];
    if (hd.z + hd.w <= zb || hd.z >= zb + ZC) continue;  // no plane of this chunk (uniform)
    int dx = gx - hd.x;
    if (dx < 0) dx += g.nx;
    if (!LANE && dx >= px) continue;  // a lane list holds only candidates that cover gx
    int dy = gy - hd.y;
    if (dy < 0) dy += g.ny;
    const T* tv = reinterpret_cast<const T*>(r + 8);
    const T* pm = tv + 6;               // monopole phi
    const T* ph = tv + 6 + stride;      // dipole phi
    const T* pd = tv + 6 + 2 * stride;  // dipole phi'
    const T mxy = pm[dx] * pm[g.pxc + dy];
    const T fm0 = tv[0] * mxy, fm1 = tv[1] * mxy, fm2 = tv[2] * mxy;
    const T fx = ph[dx], fy = ph[g.pxc + dy];
    const T wxy = fx * fy, bx = pd[dx] * fy, by = fx * pd[g.pxc + dy];
    const T tx = tv[3], ty = tv[4], tz = tv[5];
    const T a0 = by * tz, b0 = -wxy * ty;
    const T a1 = -bx * tz, b1 = wxy * tx;
    const T a2 = bx * ty - by * tx;
#pragma unroll
    for (int zz = 0; zz < ZC; ++zz) {
      const int iz = zb + zz - hd.z;
      if (iz >= 0 && iz < hd.w) {
        const T mz = pm[2 * g.pxc + iz], pz = ph[2 * g.pxc + iz], dz = pd[2 * g.pxc + iz];
        acc[zz][0] += fm0 * mz + a0 * pz + b0 * dz;
        acc[zz][1] += fm1 * mz + a1 * pz + b1 * dz;
        acc[zz][2] += fm2 * mz + a2 * pz;
      }
    }
  }
}

// the force and torque at the head of a staged record's values (16-byte aligned: records are whole
// 16-byte pieces and the values follow the two 16-byte heads), in vector loads
__device__ __forceinline__ void load6(const float* tv, float (&v)[6]) {
  const float4 a = *reinterpret_cast<const float4*>(tv);
  const float2 b = *reinterpret_cast<const float2*>(tv + 4);
  v[0] = a.x; v[1] = a.y; v[2] = a.z; v[3] = a.w; v[4] = b.x; v[5] = b.y;
}
__device__ __forceinline__ void load6(const double* tv, double (&v)[6]) {
#pragma unroll
  for (int i = 0; i < 3; ++i) {
    const double2 a = reinterpret_cast<const double2*>(tv)[i];
    v[2 * i] = a.x;
    v[2 * i + 1] = a.y;
  }
}

// Spectral-curl route with coinciding supports (m_M = m_D): each listed candidate adds F Delta_M to
// the force fields and tau Delta_D to the torque fields in one walk (six accumulators per plane).
template <typename T, int ZC, bool LANE>
__device__ __forceinline__ void spread_six_list(const Geometry& g, const uint32_t* srec, const void* wl, int nl,
                                                int rw, int gx, int gy, int zb, T (&acc)[ZC][6]) {
  const int stride = 2 * g.pxc + g.lzc;
  const int px = g.kM.px;
  for (int e = 0; e < nl; ++e) {
    const uint32_t* r = srec + (size_t)list_entry<LANE>(wl, e) * rw;
    const int4 hd = reinterpret_cast<const int4*>(r)[0];
    if (hd.z + hd.w <= zb || hd.z >= zb + ZC) continue;  // no plane of this chunk (uniform)
    int dx = gx - hd.x;
    if (dx < 0) dx += g.nx;
    if (!LANE && dx >= px) continue;  // a lane list holds only candidates that cover gx
    int dy = gy - hd.y;
    if (dy < 0) dy += g.ny;
    const T* tv = reinterpret_cast<const T*>(r + 8);
    const T* pm = tv + 6;           // monopole phi
    const T* pd = tv + 6 + stride;  // dipole phi
    const T mxy = pm[dx] * pm[g.pxc + dy], dxy = pd[dx] * pd[g.pxc + dy];
    T v[6];
    load6(tv, v);
    const T f0 = v[0] * mxy, f1 = v[1] * mxy, f2 = v[2] * mxy;
    const T t0 = v[3] * dxy, t1 = v[4] * dxy, t2 = v[5] * dxy;
#pragma unroll
    for (int zz = 0; zz < ZC; ++zz) {
      const int iz = zb + zz - hd.z;
      if (iz >= 0 && iz < hd.w) {
        const T mz = pm[2 * g.pxc + iz], dz = pd[2 * g.pxc + iz];
        acc[zz][0] += f0 * mz;
        acc[zz][1] += f1 * mz;
        acc[zz][2] += f2 * mz;
        acc[zz][3] += t0 * dz;
        acc[zz][4] += t1 * dz;
        acc[zz][5] += t2 * dz;
      }
    }
  }
}

// Bins searched around tile (bx, by) (the rbx x rby neighbourhood in (dy, dx) order, each bin at its
// first occurrence) and the prefix sums of their particle counts.  Warp 0 fills them, each lane one
// or two entries of the neighbourhood (at most 64, checked at plan creation): the counts are loaded
// all at once and summed by a warp scan.  The caller synchronises.
struct TileBins {
  int bins[64];
  int start[64];  // each bin's first entry in the sorted particle list
  int pref[65];
  int nb;
};

__device__ __forceinline__ void tile_bins(const Geometry& g, const int* __restrict__ bin_start, int bx, int by,
                                          TileBins& tb) {
  const int lane = threadIdx.x & 31;
  const unsigned below = (1u << lane) - 1u;
  const int wx = 2 * g.rbx + 1, nn = wx * (2 * g.rby + 1);
  int b[2];
#pragma unroll
  for (int h = 0; h < 2; ++h) {
    const int i = lane + 32 * h;
    b[h] = -1;
    if (i < nn) b[h] = wrap_idx(by + i / wx - g.rby, g.nby) * g.nbx + wrap_idx(bx + i % wx - g.rbx, g.nbx);
  }
  // drop an entry when an earlier entry names the same bin (small grids wrap onto themselves)
  bool keep0 = b[0] >= 0, keep1 = b[1] >= 0;
  for (int k = 0; k < 32; ++k) {
    const int o0 = __shfl_sync(0xffffffffu, b[0], k), o1 = __shfl_sync(0xffffffffu, b[1], k);
    if (k < lane && o0 == b[0]) keep0 = false;
    if (o0 == b[1] || (k < lane && o1 == b[1])) keep1 = false;
  }
  const int a0 = keep0 ? bin_start[b[0]] : 0, a1 = keep1 ? bin_start[b[1]] : 0;
  const int c0 = keep0 ? bin_start[b[0] + 1] - a0 : 0;
  const int c1 = keep1 ? bin_start[b[1] + 1] - a1 : 0;
  int s0 = c0, s1 = c1;  // inclusive scans over the lanes
#pragma unroll
  for (int off = 1; off < 32; off <<= 1) {
    const int t0 = __shfl_up_sync(0xffffffffu, s0, off), t1 = __shfl_up_sync(0xffffffffu, s1, off);
    if (lane >= off) {
      s0 += t0;
      s1 += t1;
    }
  }
  const int tot0 = __shfl_sync(0xffffffffu, s0, 31), tot1 = __shfl_sync(0xffffffffu, s1, 31);
  const unsigned m0 = __ballot_sync(0xffffffffu, keep0), m1 = __ballot_sync(0xffffffffu, keep1);
  if (keep0) {
    const int p = __popc(m0 & below);
    tb.bins[p] = b[0];
    tb.start[p] = a0;
    tb.pref[p] = s0 - c0;
  }
  if (keep1) {
    const int p = __popc(m0) + __popc(m1 & below);
    tb.bins[p] = b[1];
    tb.start[p] = a1;
    tb.pref[p] = tot0 + s1 - c1;
  }
  if (lane == 0) {
    const int nb = __popc(m0) + __popc(m1);
    tb.nb = nb;
    tb.pref[nb] = tot0 + tot1;
  }
}

// One window of the tile's candidates: the particles of the searched bins (in bin order, each bin's
// particles in index order) whose support overlaps the tile for some record head; those of rank
// [win0, win0 + kCandCap) among them go to cand[rank - win0].  Returns the number of candidates of
// all windows.  Every thread of the block (kSpreadThreads) calls it.
__device__ __forceinline__ int tile_candidates(const Geometry& g, const uint32_t* __restrict__ rec,
                                               const int* __restrict__ bin_start, const int* __restrict__ sorted,
                                               const TileBins& tb, int tx0, int ty0, int tw, int th, int win0,
                                               int* cand, int* s_warp) {
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int rw = g.rec_words;
  const int nb = tb.nb, total = tb.pref[nb];
  const int win1 = win0 + kCandCap;
  int passed = 0;  // passing candidates seen so far (uniform)
  for (int e0 = 0; e0 < total; e0 += kSpreadThreads) {
    const int e = e0 + tid;
    bool pass = false;
    int j = 0;
    if (e < total) {
      int b = 0;
      while (b + 1 < nb && tb.pref[b + 1] <= e) ++b;
      j = sorted[tb.start[b] + (e - tb.pref[b])];
      const uint32_t* r = rec + (size_t)j * rw;
      for (int K = 0; K < g.nkernels; ++K) {
        const int4 hd = reinterpret_cast<const int4*>(r)[K];
        const int px = (K == 0) ? g.kM.px : g.kD.px;
        if (hd.w > 0 && cyc_overlap(hd.x, px, tx0, tw, g.nx) && cyc_overlap(hd.y, px, ty0, th, g.ny)) pass = true;
      }
    }
    const unsigned m = __ballot_sync(0xffffffffu, pass);
    if (lane == 0) s_warp[warp] = __popc(m);
    __syncthreads();
    int woff = 0, btot = 0;
    for (int w = 0; w < kSpreadThreads / 32; ++w) {
      if (w < warp) woff += s_warp[w];
      btot += s_warp[w];
    }
    const int rank = passed + woff + __popc(m & ((1u << lane) - 1u));
    if (pass && rank >= win0 && rank < win1) cand[rank - win0] = j;
    passed += btot;
    __syncthreads();
  }
  return passed;
}

// MODE 0: forces only (3 fields); 1: spectral-curl torques (force fields, then torque fields, one
// pass each); 2: kernel-derivative torques (the force density and the half-curl sources in one pass
// over the 3 fields); 3: as 2 with coinciding supports (one list, one walk per candidate); 4: as 1
// with coinciding supports (one walk per candidate writes all six fields).
// Compiled for three resident blocks per SM in float (two in double): while one block gathers and
// stages its candidates, the others keep the SM busy.  The modes with one candidate list keep one
// list per warp in shared memory, so that three blocks fit beside kStage staged records of the
// six-field mode.
template <typename T, int MODE, int ZC>
__global__ void __launch_bounds__(kSpreadThreads, sizeof(T) == 4 ? 3 : 2)
spread_kernel(Geometry g, const uint32_t* __restrict__ rec, const int* __restrict__ bin_start,
              const int* __restrict__ sorted, const int* __restrict__ zrange, T* __restrict__ grid) {
  constexpr bool TWO = MODE == 1 || MODE == 2;  // a second list (dipole kernel of another width)
  constexpr int NL = TWO ? 2 : 1;
  extern __shared__ __align__(16) uint32_t srec[];   // g.stage_cap (<= kStage) staged records
  __shared__ TileBins s_tb;
  __shared__ int s_cand[kCandCap];
  __shared__ int s_warp[kSpreadThreads / 32];
  __shared__ int s_wl[kSpreadThreads / 32][NL][kStage];  // per-warp row lists (monopole, dipole)
  __shared__ unsigned char s_ll[kSpreadThreads / 32][NL][kLaneCap * 32];  // per-lane lists of the row lists
  const int clo = zrange[0], chi = zrange[1];
  if (chi < clo) return;
  const int bx = blockIdx.x % g.nbx, by = blockIdx.x / g.nbx;
  const int tx0 = bx * kTileX, ty0 = by * kTileY;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int gx = tx0 + (tid % kTileX), gy = ty0 + (tid / kTileX);
  const bool active = (gx < g.nx) && (gy < g.ny);
  const int tw = min(kTileX, g.nx - tx0), th = min(kTileY, g.ny - ty0);
  const int rw = g.rec_words;
  if (warp == 0) tile_bins(g, bin_start, bx, by, s_tb);
  __syncthreads();
  const size_t plane = (size_t)g.ny * 2 * g.pitch;          // T values per z plane (real rows)
  const size_t fstride = plane * g.nz;
  const size_t node = (size_t)gy * 2 * g.pitch + gx;
  // copy records [i0, i0 + cnt) of the candidate list into shared memory (16-byte pieces; records
  // are 16-byte aligned), all copies in flight at once
  auto stage = [&](int i0, int cnt) {
    const int q = rw >> 2;  // 16-byte pieces per record; a warp copies one record at a time
    for (int i = warp; i < cnt; i += kSpreadThreads / 32) {
      const uint32_t* src = rec + (size_t)s_cand[i0 + i] * rw;
      uint32_t* dst = srec + (size_t)i * rw;
      for (int w = lane; w < q; w += 32) cp_async16(dst + 4 * w, src + 4 * w);
    }
    cp_commit();
    cp_wait_all();
  };
  // rounds over windows of kCandCap passing candidates (one round unless the tile is crowded)
  for (int round = 0;; ++round) {
    const int win0 = round * kCandCap, win1 = win0 + kCandCap;
    const int passed = tile_candidates(g, rec, bin_start, sorted, s_tb, tx0, ty0, tw, th, win0, s_cand, s_warp);
    const int ncand = min(passed, win1) - win0;
    if (ncand <= 0 && round > 0) break;
    constexpr int NA = MODE == 4 ? 6 : 3;  // fields accumulated per pass
    const bool once = ncand <= g.stage_cap;
    int nl0 = 0, nl1 = 0;
    int* wl0 = s_wl[warp][0];
    int* wl1 = s_wl[warp][NL - 1];  // the one-list modes never fill or walk it
    unsigned char* ll0 = s_ll[warp][0];
    unsigned char* ll1 = s_ll[warp][NL - 1];
    int lc0 = 0, lc1 = 0;
    bool lanes = false;  // warp-uniform: walk per-lane lists instead of the row lists
    if (once) {
      stage(0, max(ncand, 0));
      __syncthreads();
      build_row_lists<TWO>(g, srec, max(ncand, 0), rw, gy, wl0, wl1, nl0, nl1);
      lc0 = build_lane_list<0>(g, srec, wl0, nl0, rw, gx, active, ll0);
      if (TWO) lc1 = build_lane_list<1>(g, srec, wl1, nl1, rw, gx, active, ll1);
      lanes = !__any_sync(0xffffffffu, lc0 > kLaneCap || lc1 > kLaneCap);
      __syncwarp();
    }
    // the candidates of list set (wl0, wl1) into the accumulators of pass K
    auto walk = [&](auto lane_tag, int K, T (&acc)[ZC][NA], int zb) {
      constexpr bool L = decltype(lane_tag)::value;
      const void* w0 = L ? static_cast<const void*>(ll0) : static_cast<const void*>(wl0);
      const void* w1 = L ? static_cast<const void*>(ll1) : static_cast<const void*>(wl1);
      const int n0 = L ? lc0 : nl0, n1 = L ? lc1 : nl1;
      (void)w1;  // the second list serves the two-pass modes only
      (void)n1;
      if constexpr (MODE == 4) {
        spread_six_list<T, ZC, L>(g, srec, w0, n0, rw, gx, gy, zb, acc);
      } else if constexpr (MODE == 3) {
        spread_fused_list<T, ZC, L>(g, srec, w0, n0, rw, gx, gy, zb, acc);
      } else if constexpr (MODE == 2) {
        spread_list<T, ZC, 0, L>(g, srec, w0, n0, rw, gx, gy, zb, acc);
        spread_curl_list<T, ZC, L>(g, srec, w1, n1, rw, gx, gy, zb, acc);
      } else {
        if (K == 0) spread_list<T, ZC, 0, L>(g, srec, w0, n0, rw, gx, gy, zb, acc);
        else spread_list<T, ZC, 1, L>(g, srec, w1, n1, rw, gx, gy, zb, acc);
      }
    };
    // the candidates of the current lists into the accumulators of pass K
    auto apply = [&](int K, T (&acc)[ZC][NA], int zb) {
      if (lanes) walk(std::true_type{}, K, acc, zb);
      else walk(std::false_type{}, K, acc, zb);
    };
    // one pass per field triple (spectral curl: force fields, then torque fields), ZC planes at a time
    constexpr int NPASS = MODE == 1 ? 2 : 1;
#pragma unroll
    for (int K = 0; K < NPASS; ++K) {
      for (int zb = clo; zb <= chi; zb += ZC) {
        T acc[ZC][NA];
#pragma unroll
        for (int zz = 0; zz < ZC; ++zz)
#pragma unroll
          for (int f = 0; f < NA; ++f) {
            T v = (T)0;
            if (round > 0 && active && zb + zz <= chi)
              v = grid[(3 * K + f) * fstride + (size_t)(zb + zz) * plane + node];
            acc[zz][f] = v;
          }
        if (!once) {
          for (int i0 = 0; i0 < ncand; i0 += g.stage_cap) {
            const int cnt = min(g.stage_cap, ncand - i0);
            __syncthreads();
            stage(i0, cnt);
            __syncthreads();
            build_row_lists<TWO>(g, srec, cnt, rw, gy, wl0, wl1, nl0, nl1);
            if (active) walk(std::false_type{}, K, acc, zb);
          }
        } else if (active) {
          apply(K, acc, zb);
        }
        if (active) {
#pragma unroll
          for (int zz = 0; zz < ZC; ++zz) {
            if (zb + zz <= chi) {
#pragma unroll
              for (int f = 0; f < NA; ++f) grid[(3 * K + f) * fstride + (size_t)(zb + zz) * plane + node] = acc[zz][f];
            }
          }
        }
      }
    }
    if (passed <= win1) break;
    __syncthreads();
  }
}

// ---------------------------------------------------------------------------------------------
// Interpolation as a tile gather, the transpose of the spread: a block owns a 32 x 8 tile of node
// columns and the candidates of the surrounding bins (the spread's lists).  Each thread reads its
// column of the occupied planes once, ZC planes at a time (coalesced rows, weighted by the
// Clenshaw-Curtis weights as loaded), and for every listed candidate whose support covers the column
// adds sum_z u(z) phi_z(z) times phi_x phi_y into that candidate's shared accumulators.  A
// particle's support overlaps at most sxn x syn tiles; each tile writes its share into the slot
// ((bx - bx0) mod nbx, (by - by0) mod nby) of a partial-sum buffer [slot][field][n] (bx0, by0: the
// tiles of the support's first node), and interp_finish_kernel adds the slots of the tiles that
// overlap the support in a fixed order.  Within a tile the columns' shares meet in shared-memory
// float atomics, whose order varies: repeated products agree to rounding, not bit for bit (the
// warp-per-particle kernels below sum in a fixed order).
// MODE 0: U from fields 0..2 (monopole); MODE 4: U and Omega from fields 0..5 with coinciding
// supports (spectral-curl torque route, m_M = m_D).
// ---------------------------------------------------------------------------------------------
// z sums of one staged candidate over the planes [zb, zb + ZC) of its support: a[f] += sum_z u phi_z
// (monopole profile for fields 0..2, dipole profile for 3..5)
template <typename T, int ZC, int NF>
__device__ __forceinline__ void interp_zsum(const Geometry& g, const uint32_t* r, int zb, const T (&u)[ZC][NF],
                                            T (&a)[NF]) {
  const int4 hd = reinterpret_cast<const int4*>(r)[0];
  if (hd.z + hd.w <= zb || hd.z >= zb + ZC) return;  // no plane of this chunk
  const int stride = 2 * g.pxc + g.lzc;
  const T* pm = reinterpret_cast<const T*>(r + 8) + 6;  // monopole phi
  const T* pd = pm + stride;                            // dipole phi (six fields)
#pragma unroll
  for (int zz = 0; zz < ZC; ++zz) {
    const int iz = zb + zz - hd.z;
    if (iz >= 0 && iz < hd.w) {
      const T mz = pm[2 * g.pxc + iz];
#pragma unroll
      for (int f = 0; f < 3; ++f) a[f] += u[zz][f] * mz;
      if (NF == 6) {
        const T dz = pd[2 * g.pxc + iz];
#pragma unroll
        for (int f = 3; f < NF; ++f) a[f] += u[zz][f] * dz;
      }
    }
  }
}

// a[f] times the candidate's x y weights at column (gx, gy), added to its shared accumulators;
// false (nothing added) when the column is outside its x support
template <typename T, int NF>
__device__ __forceinline__ bool interp_commit(const Geometry& g, const uint32_t* r, int gx, int gy, const T (&a)[NF],
                                              T* acc) {
  const int4 hd = reinterpret_cast<const int4*>(r)[0];
  const int px = g.kM.px;
  int dx = gx - hd.x;
  if (dx < 0) dx += g.nx;
  if (dx >= px) return false;
  int dy = gy - hd.y;
  if (dy < 0) dy += g.ny;
  const T* pm = reinterpret_cast<const T*>(r + 8) + 6;
  const T mxy = pm[dx] * pm[g.pxc + dy];
#pragma unroll
  for (int f = 0; f < 3; ++f) atomicAdd(&acc[f], a[f] * mxy);
  if (NF == 6) {
    const T* pd = pm + 2 * g.pxc + g.lzc;
    const T dxy = pd[dx] * pd[g.pxc + dy];
#pragma unroll
    for (int f = 3; f < NF; ++f) atomicAdd(&acc[f], a[f] * dxy);
  }
  return true;
}

// lane-list entries whose z sums a thread keeps in registers across the z chunks (one set of
// shared atomics per entry at the end instead of one per chunk)
constexpr int kInterpRegEntries = 6;

template <typename T, int MODE, int ZC>
__global__ void __launch_bounds__(kSpreadThreads)
interp_tile_kernel(Geometry g, const uint32_t* __restrict__ rec, const int* __restrict__ bin_start,
                   const int* __restrict__ sorted, const int* __restrict__ zrange, const T* __restrict__ grid,
                   const T* __restrict__ wz, T* __restrict__ part, int64_t n, int sxn, int syn,
                   int* __restrict__ status) {
  constexpr int NF = MODE == 4 ? 6 : 3;
  extern __shared__ __align__(16) uint32_t srec[];   // g.stage_cap (<= kStage) staged records
  __shared__ TileBins s_tb;
  __shared__ int s_cand[kCandCap];
  __shared__ int s_warp[kSpreadThreads / 32];
  __shared__ int s_wl[kSpreadThreads / 32][2][kStage];
  __shared__ unsigned char s_ll[kSpreadThreads / 32][2][kLaneCap * 32];
  __shared__ T s_acc[kStage][NF];  // this tile's share of each staged candidate's sums
  const int clo = zrange[0], chi = zrange[1];
  if (chi < clo) return;
  const int bx = blockIdx.x % g.nbx, by = blockIdx.x / g.nbx;
  const int tx0 = bx * kTileX, ty0 = by * kTileY;
  const int tid = threadIdx.x, warp = tid >> 5;
  const int gx = tx0 + (tid % kTileX), gy = ty0 + (tid / kTileX);
  const bool active = (gx < g.nx) && (gy < g.ny);
  const int tw = min(kTileX, g.nx - tx0), th = min(kTileY, g.ny - ty0);
  const int rw = g.rec_words;
  if (warp == 0) tile_bins(g, bin_start, bx, by, s_tb);
  __syncthreads();
  const size_t plane = (size_t)g.ny * 2 * g.pitch;
  const size_t fstride = plane * g.nz;
  const size_t node = (size_t)gy * 2 * g.pitch + gx;
  int* wl0 = s_wl[warp][0];
  int* wl1 = s_wl[warp][1];
  unsigned char* ll0 = s_ll[warp][0];
  for (int round = 0;; ++round) {
    const int win0 = round * kCandCap, win1 = win0 + kCandCap;
    const int passed = tile_candidates(g, rec, bin_start, sorted, s_tb, tx0, ty0, tw, th, win0, s_cand, s_warp);
    const int ncand = min(passed, win1) - win0;
    if (ncand <= 0) break;
    for (int i0 = 0; i0 < ncand; i0 += g.stage_cap) {
      const int cnt = min(g.stage_cap, ncand - i0);
      __syncthreads();  // the previous batch has finished with the staged records and sums
      {
        const int q = rw >> 2;
        for (int t = tid; t < cnt * q; t += kSpreadThreads) {
          const int i = t / q, w = t - i * q;
          cp_async16(srec + (size_t)i * rw + 4 * w, rec + (size_t)s_cand[i0 + i] * rw + 4 * w);
        }
        cp_commit();
      }
      for (int t = tid; t < cnt * NF; t += kSpreadThreads) s_acc[t / NF][t % NF] = (T)0;
      cp_wait_all();
      __syncthreads();
      int nl0 = 0, nl1 = 0;
      build_row_lists<false>(g, srec, cnt, rw, gy, wl0, wl1, nl0, nl1);
      const int lc0 = build_lane_list<0>(g, srec, wl0, nl0, rw, gx, active, ll0);
      const bool lanes = !__any_sync(0xffffffffu, lc0 > kLaneCap);
      __syncwarp();
      constexpr int E = kInterpRegEntries;
      T racc[E][NF];  // z sums of the first E lane-list entries, across all chunks
#pragma unroll
      for (int e = 0; e < E; ++e)
#pragma unroll
        for (int f = 0; f < NF; ++f) racc[e][f] = (T)0;
      for (int zb = clo; zb <= chi; zb += ZC) {
        T u[ZC][NF];
#pragma unroll
        for (int zz = 0; zz < ZC; ++zz) {
          const bool in = active && zb + zz <= chi;
          const T w = in ? wz[zb + zz] : (T)0;
#pragma unroll
          for (int f = 0; f < NF; ++f) u[zz][f] = in ? grid[f * fstride + (size_t)(zb + zz) * plane + node] * w : (T)0;
        }
        if (!active) continue;
        if (lanes) {
#pragma unroll
          for (int e = 0; e < E; ++e)
            if (e < lc0) interp_zsum<T, ZC, NF>(g, srec + (size_t)list_entry<true>(ll0, e) * rw, zb, u, racc[e]);
          for (int e = E; e < lc0; ++e) {  // further entries: shared atomics per chunk
            const int idx = list_entry<true>(ll0, e);
            T a[NF];
#pragma unroll
            for (int f = 0; f < NF; ++f) a[f] = (T)0;
            interp_zsum<T, ZC, NF>(g, srec + (size_t)idx * rw, zb, u, a);
            interp_commit<T, NF>(g, srec + (size_t)idx * rw, gx, gy, a, s_acc[idx]);
          }
        } else {  // the warp's row list (a lane list overflowed): shared atomics per chunk
          for (int e = 0; e < nl0; ++e) {
            const int idx = list_entry<false>(wl0, e);
            T a[NF];
#pragma unroll
            for (int f = 0; f < NF; ++f) a[f] = (T)0;
            interp_zsum<T, ZC, NF>(g, srec + (size_t)idx * rw, zb, u, a);
            interp_commit<T, NF>(g, srec + (size_t)idx * rw, gx, gy, a, s_acc[idx]);
          }
        }
      }
      if (active && lanes) {
#pragma unroll
        for (int e = 0; e < E; ++e)
          if (e < lc0) {
            const int idx = list_entry<true>(ll0, e);
            interp_commit<T, NF>(g, srec + (size_t)idx * rw, gx, gy, racc[e], s_acc[idx]);
          }
      }
      __syncthreads();
      for (int i = tid; i < cnt; i += kSpreadThreads) {
        const int4 hd = reinterpret_cast<const int4*>(srec + (size_t)i * rw)[0];
        int sx = bx - hd.x / kTileX, sy = by - hd.y / kTileY;
        if (sx < 0) sx += g.nbx;
        if (sy < 0) sy += g.nby;
        if (sx >= sxn || sy >= syn) {
          atomicOr(status, kStatInternal);
          continue;
        }
        const int64_t j = s_cand[i0 + i];
        T* dst = part + (size_t)(sy * sxn + sx) * NF * n + j;
#pragma unroll
        for (int f = 0; f < NF; ++f) dst[(size_t)f * n] = s_acc[i][f];
      }
    }
    if (passed <= win1) break;
    __syncthreads();
  }
}

// U (and Omega) of each particle: the partial sums of the tiles that overlap its support (the
// candidate test of the tile kernels), added in slot order and scaled by h^2.
template <typename T, int MODE>
__global__ void interp_finish_kernel(Geometry g, int64_t n, const uint32_t* __restrict__ rec, const T* __restrict__ part,
                                     int sxn, int syn, double* __restrict__ U, double* __restrict__ W) {
  constexpr int NF = MODE == 4 ? 6 : 3;
  const int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (j >= n) return;
  const int4 hd = reinterpret_cast<const int4*>(rec + (size_t)j * g.rec_words)[0];
  T a[NF];
#pragma unroll
  for (int f = 0; f < NF; ++f) a[f] = (T)0;
  if (hd.w > 0) {
    const int px = g.kM.px;
    const int bx0 = hd.x / kTileX, by0 = hd.y / kTileY;
    for (int sy = 0; sy < syn; ++sy) {
      const int by = (by0 + sy) % g.nby, ty0 = by * kTileY;
      if (!cyc_overlap(hd.y, px, ty0, min(kTileY, g.ny - ty0), g.ny)) continue;
      for (int sx = 0; sx < sxn; ++sx) {
        const int bx = (bx0 + sx) % g.nbx, tx0 = bx * kTileX;
        if (!cyc_overlap(hd.x, px, tx0, min(kTileX, g.nx - tx0), g.nx)) continue;
        const T* src = part + (size_t)(sy * sxn + sx) * NF * n + j;
#pragma unroll
        for (int f = 0; f < NF; ++f) a[f] += src[(size_t)f * n];
      }
    }
  }
  const double h2 = g.h * g.h;
#pragma unroll
  for (int f = 0; f < NF; ++f) {
    double* out = f < 3 ? U + 3 * j + f : W + 3 * j + (f - 3);
    if (sizeof(T) == 4) *out = widen_bits((float)a[f] * (float)h2);  // float path: widen on the integer pipe
    else *out = h2 * (double)a[f];
  }
}

// Interpolation, a warp per particle (bin order, so neighbouring warps reuse grid lines in cache):
// the warp splits into NG = 32 / LR groups of LR >= px lanes; a group walks whole x runs of the
// support rows (iz, iy), lane lx reading node x = hd.x + lx.  Rows are decoded with a multiply-shift
// (exact for rows < 2^16 / px) and UR rows are gathered before they are accumulated, so each lane
// keeps 3 UR loads in flight.
template <typename T, int LR>
__global__ void __launch_bounds__(256) interp_kernel(Geometry g, int64_t n, const uint32_t* __restrict__ rec,
                                                     const T* __restrict__ grid, const T* __restrict__ wz,
                                                     const int* __restrict__ order, double* __restrict__ U,
                                                     double* __restrict__ W) {
  constexpr int NG = 32 / LR;
  constexpr int UR = 4;
  const int64_t i = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int lane = threadIdx.x & 31;
  if (i >= n) return;
  const int64_t j = order[i];  // particles in bin order
  const uint32_t* r = rec + (size_t)j * g.rec_words;
  const T* tv = reinterpret_cast<const T*>(r + 8);
  const int lx = lane % LR, grp = lane / LR;
  const size_t rowlen = (size_t)2 * g.pitch;
  const size_t plane = (size_t)g.ny * rowlen;
  const size_t fstride = plane * g.nz;
  const int stride = 2 * g.pxc + g.lzc;
  const double h2 = g.h * g.h;
  for (int K = 0; K < g.nkernels; ++K) {
    const int4 hd = reinterpret_cast<const int4*>(r)[K];
    const int px = (K == 0) ? g.kM.px : g.kD.px;
    const T* ph = tv + 6 + K * stride;
    const bool vx = grp < NG && lx < px;
    int xi = hd.x + lx;
    if (xi >= g.nx) xi -= g.nx;
    const T phx = vx ? ph[lx] : (T)0;
    const unsigned magic = (65536u + (unsigned)px - 1u) / (unsigned)px;  // ceil(2^16 / px)
    T a0 = 0, a1 = 0, a2 = 0;
    const int rows = hd.w * px;
    const T* gbase = grid + (size_t)(3 * K) * fstride + xi;
    for (int r0 = grp; r0 < rows; r0 += NG * UR) {
      T v0[UR], v1[UR], v2[UR], wv[UR];
#pragma unroll
      for (int u = 0; u < UR; ++u) {
        const int rr = r0 + u * NG;
        v0[u] = v1[u] = v2[u] = wv[u] = (T)0;
        if (vx && rr < rows) {
          const int iz = (int)(((unsigned)rr * magic) >> 16), iy = rr - iz * px;
          const int c = hd.z + iz;
          int yi = hd.y + iy;
          if (yi >= g.ny) yi -= g.ny;
          wv[u] = ph[2 * g.pxc + iz] * wz[c] * ph[g.pxc + iy] * phx;
          const T* gp = gbase + (size_t)c * plane + (size_t)yi * rowlen;
          v0[u] = gp[0];
          v1[u] = gp[fstride];
          v2[u] = gp[2 * fstride];
        }
      }
#pragma unroll
      for (int u = 0; u < UR; ++u) {
        a0 += v0[u] * wv[u];
        a1 += v1[u] * wv[u];
        a2 += v2[u] * wv[u];
      }
    }
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) {
      a0 += __shfl_xor_sync(0xffffffffu, a0, off);
      a1 += __shfl_xor_sync(0xffffffffu, a1, off);
      a2 += __shfl_xor_sync(0xffffffffu, a2, off);
    }
    double* out = (K == 0) ? U : W;
    if (lane == 0) {
      if (sizeof(T) == 4) {  // float path: scale in float, widen on the integer pipe
        const float h2f = (float)h2;
        out[3 * j] = widen_bits((float)a0 * h2f);
        out[3 * j + 1] = widen_bits((float)a1 * h2f);
        out[3 * j + 2] = widen_bits((float)a2 * h2f);
      } else {
        out[3 * j] = h2 * (double)a0;
        out[3 * j + 1] = h2 * (double)a1;
        out[3 * j + 2] = h2 * (double)a2;
      }
    }
  }
}

// Kernel-derivative torque route: U_j = h^2 sum w_c u Delta_M and
// Omega_j = (1/2) h^2 sum w_c u x grad Delta_D (records hold the dipole phi and phi' slabs), a warp
// per particle with the row walk of interp_kernel.  FUSED (monopole and dipole supports coincide,
// m_M = m_D): one walk reads each velocity node once for both outputs; otherwise U is gathered over
// the monopole support first and Omega over the dipole support.
template <typename T, int LR, bool FUSED>
__global__ void __launch_bounds__(256, 4) interp_curl_kernel(Geometry g, int64_t n, const uint32_t* __restrict__ rec,
                                                          const T* __restrict__ grid, const T* __restrict__ wz,
                                                          const int* __restrict__ order, double* __restrict__ U,
                                                          double* __restrict__ W) {
  constexpr int NG = 32 / LR;
  constexpr int UR = 4;
  const int64_t i = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int lane = threadIdx.x & 31;
  if (i >= n) return;
  const int64_t j = order[i];
  const uint32_t* r = rec + (size_t)j * g.rec_words;
  const T* tv = reinterpret_cast<const T*>(r + 8);
  const int lx = lane % LR, grp = lane / LR;
  const size_t rowlen = (size_t)2 * g.pitch;
  const size_t plane = (size_t)g.ny * rowlen;
  const size_t fstride = plane * g.nz;
  const int stride = 2 * g.pxc + g.lzc;
  const T* pm = tv + 6;               // monopole phi
  const T* ph = tv + 6 + stride;      // dipole phi
  const T* pd = tv + 6 + 2 * stride;  // dipole phi'
  T a0 = 0, a1 = 0, a2 = 0;           // U sums
  T o0 = 0, o1 = 0, o2 = 0;           // Omega sums (without the factor 1/2)
  // walk K = 0: U over the monopole support (FUSED: skipped, done by the dipole walk);
  // K = 1: Omega over the dipole support
  for (int K = FUSED ? 1 : 0; K < 2; ++K) {
    const int4 hd = reinterpret_cast<const int4*>(r)[K];
    const int px = (K == 0) ? g.kM.px : g.kD.px;
    const bool vx = grp < NG && lx < px;
    int xi = hd.x + lx;
    if (xi >= g.nx) xi -= g.nx;
    const bool wantU = K == 0 || FUSED, wantW = K == 1;
    const T mx = (vx && wantU) ? pm[lx] : (T)0;
    const T fx = (vx && wantW) ? ph[lx] : (T)0, dxv = (vx && wantW) ? pd[lx] : (T)0;
    const unsigned magic = (65536u + (unsigned)px - 1u) / (unsigned)px;  // ceil(2^16 / px)
    const int rows = hd.w * px;
    const T* gbase = grid + xi;
    for (int r0 = grp; r0 < rows; r0 += NG * UR) {
      T v0[UR], v1[UR], v2[UR], wm[UR], gxv[UR], gyv[UR], gzv[UR];
#pragma unroll
      for (int u = 0; u < UR; ++u) {
        const int rr = r0 + u * NG;
        v0[u] = v1[u] = v2[u] = wm[u] = gxv[u] = gyv[u] = gzv[u] = (T)0;
        if (vx && rr < rows) {
          const int iz = (int)(((unsigned)rr * magic) >> 16), iy = rr - iz * px;
          const int c = hd.z + iz;
          int yi = hd.y + iy;
          if (yi >= g.ny) yi -= g.ny;
          const T w = wz[c];
          if (wantU) wm[u] = pm[2 * g.pxc + iz] * w * pm[g.pxc + iy] * mx;
          if (wantW) {
            const T pz = ph[2 * g.pxc + iz] * w, dz = pd[2 * g.pxc + iz] * w;
            const T fy = ph[g.pxc + iy], dyv = pd[g.pxc + iy];
            gxv[u] = dxv * fy * pz;
            gyv[u] = fx * dyv * pz;
            gzv[u] = fx * fy * dz;
          }
          const T* gp = gbase + (size_t)c * plane + (size_t)yi * rowlen;
          v0[u] = gp[0];
          v1[u] = gp[fstride];
          v2[u] = gp[2 * fstride];
        }
      }
#pragma unroll
      for (int u = 0; u < UR; ++u) {
        if (wantU) {
          a0 += v0[u] * wm[u];
          a1 += v1[u] * wm[u];
          a2 += v2[u] * wm[u];
        }
        if (wantW) {  // u x grad Delta
          o0 += v1[u] * gzv[u] - v2[u] * gyv[u];
          o1 += v2[u] * gxv[u] - v0[u] * gzv[u];
          o2 += v0[u] * gyv[u] - v1[u] * gxv[u];
        }
      }
    }
  }
#pragma unroll
  for (int off = 16; off > 0; off >>= 1) {
    a0 += __shfl_xor_sync(0xffffffffu, a0, off);
    a1 += __shfl_xor_sync(0xffffffffu, a1, off);
    a2 += __shfl_xor_sync(0xffffffffu, a2, off);
    o0 += __shfl_xor_sync(0xffffffffu, o0, off);
    o1 += __shfl_xor_sync(0xffffffffu, o1, off);
    o2 += __shfl_xor_sync(0xffffffffu, o2, off);
  }
  if (lane == 0) {
    const double h2 = g.h * g.h;
    if (sizeof(T) == 4) {  // float path: scale in float, widen on the integer pipe
      const float h2f = (float)h2, hh = (float)(0.5 * h2);
      U[3 * j] = widen_bits((float)a0 * h2f);
      U[3 * j + 1] = widen_bits((float)a1 * h2f);
      U[3 * j + 2] = widen_bits((float)a2 * h2f);
      W[3 * j] = widen_bits((float)o0 * hh);
      W[3 * j + 1] = widen_bits((float)o1 * hh);
      W[3 * j + 2] = widen_bits((float)o2 * hh);
    } else {
      U[3 * j] = h2 * (double)a0;
      U[3 * j + 1] = h2 * (double)a1;
      U[3 * j + 2] = h2 * (double)a2;
      W[3 * j] = 0.5 * h2 * (double)o0;
      W[3 * j + 1] = 0.5 * h2 * (double)o1;
      W[3 * j + 2] = 0.5 * h2 * (double)o2;
    }
  }
}

// Spectral-curl route with coinciding supports (m_M = m_D): one walk over the common support reads
// the velocity (fields 0..2) and the half-curl (fields 3..5) of each node and returns
// U_j = h^2 sum w_c u Delta_M and Omega_j = h^2 sum w_c omega Delta_D (the row walk of interp_kernel).
template <typename T, int LR>
__global__ void __launch_bounds__(256) interp_pair_kernel(Geometry g, int64_t n, const uint32_t* __restrict__ rec,
                                                          const T* __restrict__ grid, const T* __restrict__ wz,
                                                          const int* __restrict__ order, double* __restrict__ U,
                                                          double* __restrict__ W) {
  constexpr int NG = 32 / LR;
  constexpr int UR = 4;
  const int64_t i = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int lane = threadIdx.x & 31;
  if (i >= n) return;
  const int64_t j = order[i];
  const uint32_t* r = rec + (size_t)j * g.rec_words;
  const T* tv = reinterpret_cast<const T*>(r + 8);
  const int lx = lane % LR, grp = lane / LR;
  const size_t rowlen = (size_t)2 * g.pitch;
  const size_t plane = (size_t)g.ny * rowlen;
  const size_t fstride = plane * g.nz;
  const int stride = 2 * g.pxc + g.lzc;
  const T* pm = tv + 6;           // monopole phi
  const T* pd = tv + 6 + stride;  // dipole phi
  const int4 hd = reinterpret_cast<const int4*>(r)[0];
  const int px = g.kM.px;
  const bool vx = grp < NG && lx < px;
  int xi = hd.x + lx;
  if (xi >= g.nx) xi -= g.nx;
  const T mx = vx ? pm[lx] : (T)0, dxw = vx ? pd[lx] : (T)0;
  const unsigned magic = (65536u + (unsigned)px - 1u) / (unsigned)px;  // ceil(2^16 / px)
  const int rows = hd.w * px;
  const T* gbase = grid + xi;
  T a0 = 0, a1 = 0, a2 = 0, o0 = 0, o1 = 0, o2 = 0;
  for (int r0 = grp; r0 < rows; r0 += NG * UR) {
    T v[6][UR], wm[UR], wd[UR];
#pragma unroll
    for (int u = 0; u < UR; ++u) {
      const int rr = r0 + u * NG;
#pragma unroll
      for (int f = 0; f < 6; ++f) v[f][u] = (T)0;
      wm[u] = wd[u] = (T)0;
      if (vx && rr < rows) {
        const int iz = (int)(((unsigned)rr * magic) >> 16), iy = rr - iz * px;
        const int c = hd.z + iz;
        int yi = hd.y + iy;
        if (yi >= g.ny) yi -= g.ny;
        const T w = wz[c];
        wm[u] = pm[2 * g.pxc + iz] * w * pm[g.pxc + iy] * mx;
        wd[u] = pd[2 * g.pxc + iz] * w * pd[g.pxc + iy] * dxw;
        const T* gp = gbase + (size_t)c * plane + (size_t)yi * rowlen;
#pragma unroll
        for (int f = 0; f < 6; ++f) v[f][u] = gp[f * fstride];
      }
    }
#pragma unroll
    for (int u = 0; u < UR; ++u) {
      a0 += v[0][u] * wm[u];
      a1 += v[1][u] * wm[u];
      a2 += v[2][u] * wm[u];
      o0 += v[3][u] * wd[u];
      o1 += v[4][u] * wd[u];
      o2 += v[5][u] * wd[u];
    }
  }
#pragma unroll
  for (int off = 16; off > 0; off >>= 1) {
    a0 += __shfl_xor_sync(0xffffffffu, a0, off);
    a1 += __shfl_xor_sync(0xffffffffu, a1, off);
    a2 += __shfl_xor_sync(0xffffffffu, a2, off);
    o0 += __shfl_xor_sync(0xffffffffu, o0, off);
    o1 += __shfl_xor_sync(0xffffffffu, o1, off);
    o2 += __shfl_xor_sync(0xffffffffu, o2, off);
  }
  if (lane == 0) {
    const double h2 = g.h * g.h;
    if (sizeof(T) == 4) {  // float path: scale in float, widen on the integer pipe
      const float h2f = (float)h2;
      U[3 * j] = widen_bits((float)a0 * h2f);
      U[3 * j + 1] = widen_bits((float)a1 * h2f);
      U[3 * j + 2] = widen_bits((float)a2 * h2f);
      W[3 * j] = widen_bits((float)o0 * h2f);
      W[3 * j + 1] = widen_bits((float)o1 * h2f);
      W[3 * j + 2] = widen_bits((float)o2 * h2f);
    } else {
      U[3 * j] = h2 * (double)a0;
      U[3 * j + 1] = h2 * (double)a1;
      U[3 * j + 2] = h2 * (double)a2;
      W[3 * j] = h2 * (double)o0;
      W[3 * j + 1] = h2 * (double)o1;
      W[3 * j + 2] = h2 * (double)o2;
    }
  }
}

// ---------------------------------------------------------------------------------------------
// Interpolation with the grid staged in shared memory (float, supports of at most 6 nodes): a
// block per particle bin.  The particles of a bin (32 x 8 nodes by position) have their supports'
// first nodes within 33 x 9 of each other, so their supports lie in a region of at most 38 x 14
// node columns; the block brings that region of the occupied planes into shared memory, four planes
// at a time, and each warp gathers its particles from there: lane group g (6 x-lanes) takes plane
// g of the four, walks the 6 support rows of that plane and adds the 6 fields (U from fields 0..2
// with the monopole weights, Omega from fields 3..5 with the dipole weights; forces only: U from
// fields 0..2).  Each of 15 gather warps holds the sums of its 3 particles of a batch of 45 across
// the chunks and reduces them over its lanes at the end of the batch.
// Staging: where the region does not cross the periodic boundary, one TMA box load per chunk
// (44 x 14 x 4 x fields of the grid's tensor map) into one of three buffers, issued by a sixteenth
// warp: a buffer's `full` barrier completes with the load's bytes, its `empty` barrier when all
// gather warps have read it, and the producer waits for `empty` before loading the next chunk into
// it, so a gather warp waits only for the chunk it needs next.  Each wait is bounded (about a
// second; on expiry the block records kStatTimeout, every role leaves its loop, and the producer
// waits again, bounded, for its loads in flight before the block exits).  At the boundary the
// block copies the wrapped rows with 16-byte cp.async pieces instead (block-wide barriers).  Where a bin's
// region would not fit (it cannot with the bins' construction, but the kernel checks) the block
// gathers from global memory with the same lane walk.
// Shared layout per buffer: [field][plane of the chunk][row (14)][44]: planes 616 values apart, 8
// banks apart modulo 32, so that the four lane groups reading the same (row, column) of four
// planes hit 24 distinct banks.
// ---------------------------------------------------------------------------------------------
constexpr int kIsPX = 6;                    // support width the staged kernel handles
constexpr int kIsGroups = 4;                // lane groups = planes per chunk
constexpr int kIsSX = 44;                   // staged row length (values)
constexpr int kIsPieces = kIsSX / 4;        // 16-byte pieces per row
constexpr int kIsRows = 14;                 // staged rows per plane (9 first-node rows + 5)
constexpr int kIsPS = kIsSX * kIsRows;      // plane stride (values)
constexpr int kIsFS = kIsGroups * kIsPS;    // field stride (values)
constexpr int kIsSlots = 3;                 // particles per warp per batch
constexpr int kIsThreads = 512;
constexpr int kIsWarps = kIsThreads / 32;
constexpr int kIsGatherWarps = kIsWarps - 1;  // the last warp issues the TMA loads
constexpr int kIsBatch = kIsGatherWarps * kIsSlots;
static_assert(kIsPS % 32 == 8 && (kIsSX * 4) % 16 == 0, "staged plane layout");
static_assert(kIsGroups * kIsPX <= 32, "lane groups");

constexpr int kIsZT = 64;  // z weights of a particle's table (records with more z slots: not staged)

// a gather warp's table of one particle of the batch: the staged offset of its first support node,
// its z support, and its weights (the z weights times the Clenshaw-Curtis weights of the planes)
struct __align__(16) IsSlot {
  int base, z0, zn, pad;
  float mx[8], dx[8], my[8], dy[8];
  float mz[kIsZT], dz[kIsZT];
};

__host__ __device__ constexpr size_t interp_stage_buf(int nf) { return (size_t)nf * kIsFS * sizeof(float); }
constexpr int kIsBufs = 3;  // chunk buffers: TMA loads in flight while the warps read one
__host__ __device__ constexpr size_t interp_stage_smem(int nf) { return kIsBufs * interp_stage_buf(nf) + 128; }

// offset of node v from t0 on a periodic axis of n nodes, in (-n/2, n/2]
__device__ __forceinline__ int rel_node(int v, int t0, int n) {
  int d = v - t0;
  if (2 * d > n) d -= n;
  else if (2 * d <= -n) d += n;
  return d;
}

__device__ __forceinline__ void is_bar_init(uint64_t* bar, unsigned count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;\n" ::"r"(smem_u32(bar)), "r"(count) : "memory");
}
__device__ __forceinline__ void is_arrive(uint64_t* bar) {
  asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];\n" ::"r"(smem_u32(bar)) : "memory");
}
__device__ __forceinline__ void is_expect_tx(uint64_t* bar, unsigned bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;\n" ::"r"(smem_u32(bar)), "r"(bytes) : "memory");
}
// bounded wait for the phase with the given parity; false after about 2^31 cycles, or once the
// block's failure flag (if given) is raised
__device__ __forceinline__ bool is_wait(uint64_t* bar, unsigned parity, volatile int* fail) {
  const long long t0 = clock64();
  for (;;) {
    unsigned done;
    asm volatile(
        "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}\n"
        : "=r"(done)
        : "r"(smem_u32(bar)), "r"(parity)
        : "memory");
    if (done) return true;
    if (fail && *fail) return false;
    if (clock64() - t0 > (1LL << 31)) return false;
  }
}
__device__ __forceinline__ void is_tma_4d(void* dst, const CUtensorMap* map, int x, int y, int z, int f, uint64_t* bar) {
  asm volatile(
      "cp.async.bulk.tensor.4d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3, %4, %5}], "
      "[%6];\n" ::"r"(smem_u32(dst)),
      "l"(reinterpret_cast<uint64_t>(map)), "r"(x), "r"(y), "r"(z), "r"(f), "r"(smem_u32(bar))
      : "memory");
}

template <int NF>
__global__ void __launch_bounds__(kIsThreads, 1)
interp_stage_kernel(const __grid_constant__ CUtensorMap tmap, int use_tma, Geometry g, const uint32_t* __restrict__ rec,
                    const int* __restrict__ bin_start, const int* __restrict__ sorted, const float* __restrict__ grid,
                    const float* __restrict__ wz, double* __restrict__ U, double* __restrict__ W, int force_global,
                    int* __restrict__ status) {
  constexpr int PX = kIsPX, NG = kIsGroups, ZC = kIsGroups, SX = kIsSX, FS = kIsFS, PW = kIsSlots;
  constexpr int GW = kIsGatherWarps;
  constexpr int BUFV = NF * kIsFS;  // values per chunk buffer
  extern __shared__ __align__(128) unsigned char is_raw[];
  // two chunk buffers, 128-byte aligned (TMA destinations)
  float* const sg = reinterpret_cast<float*>(is_raw + ((128u - (smem_u32(is_raw) & 127u)) & 127u));
  __shared__ __align__(8) uint64_t s_full[kIsBufs], s_empty[kIsBufs];
  __shared__ int s_b[6];           // bounds: ox min/max, oy min/max, z begin/end
  __shared__ int s_xo[kIsSX];      // wrapped x of each staged column (cp.async path)
  __shared__ int s_yo[kIsRows];    // wrapped y of each staged row times the row length
  __shared__ int s_fail;           // a bounded wait ran out
  __shared__ IsSlot s_slot[kIsGatherWarps][kIsSlots];
  const int b = blockIdx.x;
  const int p0 = bin_start[b], cnt = bin_start[b + 1] - p0;
  if (cnt <= 0) return;
  const int tx0 = (b % g.nbx) * kTileX, ty0 = (b / g.nbx) * kTileY;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int grp = lane / PX, lx = lane - grp * PX;
  const bool lane_on = grp < NG;
  const int rw = g.rec_words, stride = 2 * g.pxc + g.lzc, px = g.kM.px;
  const int rowlen = 2 * g.pitch;
  const size_t plane = (size_t)g.ny * rowlen, fstride = plane * g.nz;
  volatile int* fail_flag = &s_fail;
  if (tid < 6) s_b[tid] = (tid & 1) ? INT_MIN : INT_MAX;
  if (tid == 0) s_fail = 0;
  __syncthreads();
  for (int i = tid; i < cnt; i += kIsThreads) {
    const int4 hd = *reinterpret_cast<const int4*>(rec + (size_t)sorted[p0 + i] * rw);
    if (hd.w <= 0) continue;
    const int ox = rel_node(hd.x, tx0, g.nx), oy = rel_node(hd.y, ty0, g.ny);
    atomicMin(&s_b[0], ox);
    atomicMax(&s_b[1], ox);
    atomicMin(&s_b[2], oy);
    atomicMax(&s_b[3], oy);
    atomicMin(&s_b[4], hd.z);
    atomicMax(&s_b[5], hd.z + hd.w);
  }
  __syncthreads();
  const int zlo = s_b[4], zhi = s_b[5];
  const bool any = zhi > zlo;
  // staged region: columns [xlo4, xlo4 + SX) (xlo4 = first support column rounded down to a
  // 16-byte piece), rows [ylo, ylo + rh)
  const int xlo = any ? tx0 + s_b[0] : 0;
  const int xlo4 = xlo >= 0 ? (xlo & ~3) : -((-xlo + 3) & ~3);
  const int xoff = xlo4 - tx0;
  const int oymin = any ? s_b[2] : 0;
  const int ylo = ty0 + oymin;
  const int rh = any ? s_b[3] - oymin + PX : 0;
  const bool staged = any && !force_global && (s_b[1] + PX - xoff <= SX) && (rh <= kIsRows) &&
                      (g.nx % 4 == 0) && (g.kM.px <= PX);
  // TMA where the columns and rows read lie inside the grid (no periodic wrap)
  const bool tma = staged && use_tma && xlo4 >= 0 && tx0 + s_b[1] + PX <= g.nx && ylo >= 0 && ylo + rh <= g.ny;
  if (staged && !tma) {
    if (tid < SX) {
      int x = (xlo4 + tid) % g.nx;
      s_xo[tid] = x < 0 ? x + g.nx : x;
    }
    if (tid < kIsRows) {
      int y = (ylo + tid) % g.ny;
      s_yo[tid] = (y < 0 ? y + g.ny : y) * rowlen;
    }
  }
  if (tma && tid == 0) {
    for (int i = 0; i < kIsBufs; ++i) {
      is_bar_init(&s_full[i], 1);
      is_bar_init(&s_empty[i], GW);
    }
    asm volatile("fence.mbarrier_init.release.cluster;\n" ::: "memory");
  }
  __syncthreads();
  const float h2f = (float)(g.h * g.h);
  const int nch = staged ? (zhi - zlo + ZC - 1) / ZC : 1;
  const int nbatch = (cnt + kIsBatch - 1) / kIsBatch;
  const int total = nbatch * nch;  // (batch, chunk) steps
  float acc[PW][NF];
  auto zero_acc = [&]() {
#pragma unroll
    for (int q = 0; q < PW; ++q)
#pragma unroll
      for (int f = 0; f < NF; ++f) acc[q][f] = 0.f;
  };
  // this warp's tables of its particles of `batch` (warp-private: __syncwarp publishes them)
  auto fill_tables = [&](int batch) {
#pragma unroll
    for (int q = 0; q < PW; ++q) {
      const int i = batch * kIsBatch + warp + GW * q;
      if (i >= cnt) continue;  // warp-uniform
      IsSlot& t = s_slot[warp][q];
      const uint32_t* r = rec + (size_t)sorted[p0 + i] * rw;
      const int4 hd = *reinterpret_cast<const int4*>(r);
      const float* pm = reinterpret_cast<const float*>(r + 8) + 6;
      const float* pd = pm + stride;
      if (lane == 0) {
        t.base = (rel_node(hd.y, ty0, g.ny) - oymin) * SX + (rel_node(hd.x, tx0, g.nx) - xoff);
        t.z0 = hd.z;
        t.zn = hd.w;
      }
      if (lane < 8) {  // zero past the support: those lanes and rows add nothing
        const bool on = lane < px;
        t.mx[lane] = on ? pm[lane] : 0.f;
        t.my[lane] = on ? pm[g.pxc + lane] : 0.f;
        t.dx[lane] = (NF == 6 && on) ? pd[lane] : 0.f;
        t.dy[lane] = (NF == 6 && on) ? pd[g.pxc + lane] : 0.f;
      }
      for (int e = lane; e < hd.w; e += 32) {
        const float wc = wz[hd.z + e];
        t.mz[e] = pm[2 * g.pxc + e] * wc;
        t.dz[e] = NF == 6 ? pd[2 * g.pxc + e] * wc : 0.f;
      }
    }
    __syncwarp();
  };
  // this warp's particles of `batch` over the staged planes [zb, zb + ZC) of buffer sb
  auto gather_staged = [&](const float* sb, int batch, int zb) {
#pragma unroll
    for (int q = 0; q < PW; ++q) {
      const int i = batch * kIsBatch + warp + GW * q;
      if (i >= cnt || !lane_on) continue;
      const IsSlot& t = s_slot[warp][q];
      const int4 head = *reinterpret_cast<const int4*>(&t.base);  // base, z0, zn in one load
      const int iz = zb + grp - head.y;
      if (iz < 0 || iz >= head.z) continue;
      const float mzx = t.mz[iz] * t.mx[lx];
      const float dzx = NF == 6 ? t.dz[iz] * t.dx[lx] : 0.f;
      const float* sp = sb + grp * kIsPS + head.x + lx;
      // the row weights (PX = 6) in vector loads: the table rows are 16-byte aligned
      static_assert(PX == 6, "row weights loaded as 4 + 2");
      const float4 my4 = *reinterpret_cast<const float4*>(t.my);
      const float2 my2 = *reinterpret_cast<const float2*>(t.my + 4);
      const float myv[PX] = {my4.x, my4.y, my4.z, my4.w, my2.x, my2.y};
      float dyv[PX] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
      if (NF == 6) {
        const float4 dy4 = *reinterpret_cast<const float4*>(t.dy);
        const float2 dy2 = *reinterpret_cast<const float2*>(t.dy + 4);
        dyv[0] = dy4.x; dyv[1] = dy4.y; dyv[2] = dy4.z; dyv[3] = dy4.w; dyv[4] = dy2.x; dyv[5] = dy2.y;
      }
#pragma unroll
      for (int iy = 0; iy < PX; ++iy) {
        const float wm = mzx * myv[iy];
#pragma unroll
        for (int f = 0; f < 3; ++f) acc[q][f] += sp[f * FS + iy * SX] * wm;
        if (NF == 6) {
          const float wd = dzx * dyv[iy];
#pragma unroll
          for (int f = 3; f < NF; ++f) acc[q][f] += sp[f * FS + iy * SX] * wd;
        }
      }
    }
  };
  // sums over the warp's lanes; lane 0 writes U (and Omega) of each of its particles of `batch`
  auto finish = [&](int batch) {
#pragma unroll
    for (int q = 0; q < PW; ++q) {
      const int i = batch * kIsBatch + warp + GW * q;
      if (i >= cnt) continue;  // warp-uniform
#pragma unroll
      for (int f = 0; f < NF; ++f)
#pragma unroll
        for (int off = 16; off > 0; off >>= 1) acc[q][f] += __shfl_xor_sync(0xffffffffu, acc[q][f], off);
      if (lane == 0) {
        const int64_t j = sorted[p0 + i];
#pragma unroll
        for (int f = 0; f < 3; ++f) U[3 * j + f] = widen_bits(acc[q][f] * h2f);
        if (NF == 6) {
#pragma unroll
          for (int f = 0; f < 3; ++f) W[3 * j + f] = widen_bits(acc[q][3 + f] * h2f);
        }
      }
    }
  };
  if (tma) {
    constexpr unsigned kBoxBytes = (unsigned)interp_stage_buf(NF);
    if (warp == GW) {
      // producer: the TMA load of each step's chunk into buffer step mod kIsBufs once the gather
      // warps have released the buffer's previous contents (its use u - 1)
      if (lane == 0) {
        int issued = 0, bb = 0, kz = 0;
        unsigned u = 0;  // use of buffer bb
        for (int step = 0; step < total; ++step) {
          if (step >= kIsBufs && !is_wait(&s_empty[bb], (u - 1u) & 1u, fail_flag)) {
            if (!*fail_flag) atomicOr(status, kStatTimeout);
            *fail_flag = 1;
            break;
          }
          if (*fail_flag) break;
          asm volatile("fence.proxy.async.shared::cta;\n" ::: "memory");  // generic reads of the buffer came first
          is_expect_tx(&s_full[bb], kBoxBytes);
          is_tma_4d(sg + bb * BUFV, &tmap, xlo4, ylo, zlo + kz * ZC, 0, &s_full[bb]);
          ++issued;
          if (++kz == nch) kz = 0;
          if (++bb == kIsBufs) {
            bb = 0;
            ++u;
          }
        }
        // loads still in flight (a stop): wait, bounded, for the last one of each buffer
        for (int st = issued - kIsBufs < 0 ? 0 : issued - kIsBufs; st < issued; ++st)
          is_wait(&s_full[st % kIsBufs], (unsigned)(st / kIsBufs) & 1u, nullptr);
      }
    } else {
      int batch = 0, k = 0, bb = 0;
      unsigned u = 0;
      for (int step = 0; step < total; ++step) {
        if (k == 0) {
          zero_acc();
          fill_tables(batch);
        }
        if (!is_wait(&s_full[bb], u & 1u, fail_flag)) {
          if (!*fail_flag) atomicOr(status, kStatTimeout);
          *fail_flag = 1;
          break;
        }
        gather_staged(sg + bb * BUFV, batch, zlo + k * ZC);
        __syncwarp();
        if (lane == 0) is_arrive(&s_empty[bb]);
        if (k == nch - 1) finish(batch);
        if (++bb == kIsBufs) {
          bb = 0;
          ++u;
        }
        if (++k == nch) {
          k = 0;
          ++batch;
        }
      }
    }
    __syncthreads();
    return;
  }
  for (int step = 0; step < total; ++step) {
    const int batch = step / nch, k = step - batch * nch;
    if (k == 0) {
      zero_acc();
      if (staged && warp < GW) fill_tables(batch);
    }
    float* sb = sg + (step & 1) * BUFV;
    if (staged) {
      __syncthreads();  // the readers of this buffer two steps ago are done
      const int zb = zlo + k * ZC;
      // rows (f, zz, yy) of the chunk: a warp copies two rows per step (22 lanes, 11 pieces each)
      const int sub = lane / kIsPieces, pc = lane - sub * kIsPieces;
      if (sub < 2) {
        for (int r = 2 * warp + sub; r < NF * ZC * kIsRows; r += 2 * kIsWarps) {
          const int yy = r % kIsRows, zz = (r / kIsRows) % ZC, f = r / (kIsRows * ZC);
          if (yy >= rh || zb + zz >= zhi) continue;
          const float* src = grid + (size_t)f * fstride + (size_t)(zb + zz) * plane + s_yo[yy] + s_xo[4 * pc];
          cp_async16(sb + f * FS + zz * kIsPS + yy * SX + 4 * pc, src);
        }
      }
      cp_commit();
      cp_wait_all();
      __syncthreads();
      if (warp < GW) gather_staged(sb, batch, zb);
    } else if (any && warp < GW) {
      // global-memory gather with the same lane walk (planes hd.z + g, g + NG, ...)
#pragma unroll
      for (int q = 0; q < PW; ++q) {
        const int i = batch * kIsBatch + warp + GW * q;
        if (i >= cnt || !lane_on) continue;
        const uint32_t* r = rec + (size_t)sorted[p0 + i] * rw;
        const int4 hd = *reinterpret_cast<const int4*>(r);
        const float* pm = reinterpret_cast<const float*>(r + 8) + 6;
        const float* pd = pm + stride;
        int x = hd.x + lx;
        if (x >= g.nx) x -= g.nx;
        const bool xon = lx < px;
        for (int iz = grp; iz < hd.w; iz += NG) {
          const int c = hd.z + iz;
          const float wc = wz[c];
          const float mzx = xon ? pm[2 * g.pxc + iz] * wc * pm[lx] : 0.f;
          const float dzx = (NF == 6 && xon) ? pd[2 * g.pxc + iz] * wc * pd[lx] : 0.f;
          for (int iy = 0; iy < px; ++iy) {
            int y = hd.y + iy;
            if (y >= g.ny) y -= g.ny;
            const float* gp = grid + (size_t)c * plane + (size_t)y * rowlen + (xon ? x : 0);
            const float wm = mzx * pm[g.pxc + iy];
#pragma unroll
            for (int f = 0; f < 3; ++f) acc[q][f] += gp[(size_t)f * fstride] * wm;
            if (NF == 6) {
              const float wd = dzx * pd[g.pxc + iy];
#pragma unroll
              for (int f = 3; f < NF; ++f) acc[q][f] += gp[(size_t)f * fstride] * wd;
            }
          }
        }
      }
    }
    if (k == nch - 1 && warp < GW) finish(batch);
  }
}

}  // namespace

// ---------------------------------------------------------------------------------------------
// host side: kernel constants and the particle-side geometry
// ---------------------------------------------------------------------------------------------

// Integral of exp(beta (sqrt(1 - (t/alpha)^2) - 1)) over [-alpha, alpha] (the normalisation of
// Eq. 54), by 128-point Gauss-Legendre quadrature after t = alpha sin(theta), which leaves the
// smooth integrand alpha exp(beta (cos(theta) - 1)) cos(theta).  Nodes by Newton iteration on the
// Legendre three-term recurrence; no heap use (the allocation-free spread calls this too).
double es_norm(double alpha, double beta) {
  const int n = 128;
  double s = 0.0;
  for (int i = 0; i < n; ++i) {
    double z = cos(M_PI * (i + 0.75) / (n + 0.5));
    double dp = 0.0;
    for (int it = 0; it < 100; ++it) {
      double p0 = 1.0, p1 = z;
      for (int k = 2; k <= n; ++k) {
        const double p2 = ((2.0 * k - 1.0) * z * p1 - (k - 1.0) * p0) / k;
        p0 = p1;
        p1 = p2;
      }
      dp = n * (z * p1 - p0) / (z * z - 1.0);  // P_n'(z) from P_n = p1, P_{n-1} = p0
      const double dz = p1 / dp;
      z -= dz;
      if (fabs(dz) < 1e-16) break;
    }
    const double w = 2.0 / ((1.0 - z * z) * dp * dp);
    const double th = 0.5 * M_PI * z;
    s += w * exp(beta * (cos(th) - 1.0)) * cos(th);
  }
  return alpha * 0.5 * M_PI * s;
}

// Truncation point of the derivative kernel: with v = (t/alpha)^2, |phi'| is stationary where
// beta v sqrt(1 - v) = 1.  The left side rises from 0 to 2/(3 sqrt 3) at v = 2/3 and falls to 0 at
// v = 1, so for beta > 3 sqrt(3)/2 the larger root, in (2/3, 1), is the minimum of |phi'| before
// it blows up at the support edge.  Bisection; -1 when there is no interior minimum.
double es_deriv_cut(double alpha, double beta) {
  if (!(beta * (2.0 / 3.0) * sqrt(1.0 / 3.0) > 1.0)) return -1.0;
  double lo = 2.0 / 3.0, hi = 1.0;
  for (int it = 0; it < 200 && hi - lo > 1e-17; ++it) {
    const double mid = 0.5 * (lo + hi);
    if (beta * mid * sqrt(1.0 - mid) - 1.0 > 0.0) lo = mid; else hi = mid;
  }
  return alpha * sqrt(0.5 * (lo + hi));
}

dps_status particle_geometry(Geometry& g, const dps_kernel_params* kp, int tsize) {
  const int route = kp->with_torque;
  if (route < DPS_TORQUE_NONE || route > DPS_TORQUE_KERNEL_DERIVATIVE) return DPS_ERR_INVALID_ARG;
  const bool torque = route != DPS_TORQUE_NONE;
  auto bad_kernel = [&](int m, double beta) {
    return m < 2 || m > kMaxM || !(beta > 0) || !isfinite(beta) || m + 1 > g.nx / 2 || m + 1 > g.ny / 2;
  };
  if (bad_kernel(kp->m_M, kp->beta_M) || (torque && bad_kernel(kp->m_D, kp->beta_D))) return DPS_ERR_INVALID_ARG;
  g.with_torque = torque ? 1 : 0;
  g.spectral_curl = route == DPS_TORQUE_SPECTRAL_CURL ? 1 : 0;
  g.torque_deriv = route == DPS_TORQUE_KERNEL_DERIVATIVE ? 1 : 0;
  g.nfields = g.spectral_curl ? 6 : 3;
  g.nkernels = torque ? 2 : 1;
  g.nslabs = g.nkernels + g.torque_deriv;
  auto setk = [&](EsKernel& k, int m, double beta) {
    k.alpha = 0.5 * m * g.h;
    k.beta = beta;
    k.inv_norm = 1.0 / es_norm(k.alpha, beta);
    k.cut = 0.0;
    k.px = m + 1;
    k.inv_alpha_f = (float)(1.0 / k.alpha);
    k.beta_f = (float)beta;
    k.inv_norm_f = (float)k.inv_norm;
    k.beta_over_alpha_f = (float)(beta / k.alpha);
  };
  setk(g.kM, kp->m_M, kp->beta_M);
  if (torque) setk(g.kD, kp->m_D, kp->beta_D); else g.kD = g.kM;
  if (g.torque_deriv) {
    g.kD.cut = es_deriv_cut(g.kD.alpha, g.kD.beta);
    if (!(g.kD.cut > 0.0)) return DPS_ERR_INVALID_ARG;
  }
  const double amax = std::max(g.kM.alpha, torque ? g.kD.alpha : 0.0);
  if (g.mode == DPS_SLIT && g.H < 2.0 * amax) return DPS_ERR_INVALID_ARG;
  if (g.mode == DPS_FREE && g.H <= 2.0 * amax) return DPS_ERR_INVALID_ARG;
  g.pxc = std::max(g.kM.px, torque ? g.kD.px : 0);
  // z slots: most Chebyshev nodes inside any closed window of length 2 alpha (plus margin)
  int best = 0;
  for (int c = 0; c < g.nz; ++c) {
    const double zc0 = g.zmin + 0.5 * g.H * (1.0 + cos(M_PI * c / (g.nz - 1)));
    int cnt = 0;
    for (int q = 0; q < g.nz; ++q) {
      const double zq = g.zmin + 0.5 * g.H * (1.0 + cos(M_PI * q / (g.nz - 1)));
      if (zq <= zc0 && zq >= zc0 - 2.0 * amax * (1.0 + 1e-9) - 1e-12 * g.H) ++cnt;
    }
    best = std::max(best, cnt);
  }
  g.lzc = std::min(g.nz, best + 2);
  const int tvals = 6 + g.nslabs * (2 * g.pxc + g.lzc);
  g.rec_words = (8 + tvals * tsize + 3) / 4 * 4;
  g.nbx = (g.nx + kTileX - 1) / kTileX;
  g.nby = (g.ny + kTileY - 1) / kTileY;
  g.rbx = (g.pxc + kTileX - 1) / kTileX + ((g.nx % kTileX) ? 1 : 0);
  g.rby = (g.pxc + kTileY - 1) / kTileY + ((g.ny % kTileY) ? 1 : 0);
  if ((2 * g.rbx + 1) * (2 * g.rby + 1) > 64) return DPS_ERR_INVALID_ARG;
  return DPS_OK;
}

template <typename T>
void launch_records(const Plan& p, int64_t n, const double* pos, const double* F, const double* Tq,
                    cudaStream_t s) {
  if (n <= 0) return;
  const int threads = p.g.rec_threads > 0 ? p.g.rec_threads : 128;
  const unsigned blocks = (unsigned)((n + threads - 1) / threads);
  if (p.g.rec_threads > 0)
    records_kernel<T, true><<<blocks, threads, (size_t)threads * p.g.rec_words * sizeof(uint32_t), s>>>(
        p.g, n, pos, F, Tq, p.tab.zc, p.records, p.bin_of, p.bin_count, p.zrange, p.status);
  else
    records_kernel<T, false><<<blocks, threads, 0, s>>>(p.g, n, pos, F, Tq, p.tab.zc, p.records, p.bin_of,
                                                        p.bin_count, p.zrange, p.status);
}

void launch_bins(const Plan& p, int64_t n, cudaStream_t s) {
  const int nbins = p.g.nbx * p.g.nby;
  bin_scan_kernel<<<1, 1024, 0, s>>>(p.bin_count, p.bin_start, p.bin_cursor, nbins);
  if (n > 0) {
    const int threads = 256;
    bin_scatter_kernel<<<(unsigned)((n + threads - 1) / threads), threads, 0, s>>>(n, p.bin_of, p.bin_cursor,
                                                                                  p.sorted);
    bin_sort_kernel<<<(unsigned)((nbins + 127) / 128), 128, 0, s>>>(p.bin_start, p.sorted, nbins);
  }
}

constexpr int kZC6F = 16, kZC6D = 8, kZC3F = 16, kZC3D = 8;  // z chunk of a pass: 3 fields x ZC accumulators
constexpr int kZCSF = 8, kZCSD = 4;                            // six fields at once: 6 x ZC accumulators

template <typename T>
size_t spread_smem(const Plan& p) {
  return (size_t)p.g.stage_cap * p.g.rec_words * sizeof(uint32_t);
}

// dynamic shared-memory limit of the spreading kernels, raised at plan creation (never at launch,
// so that applies can be captured into graphs), and the records staged at a time: kStage, or fewer
// when that many large records (wide kernels, many z slots, three slabs) would not fit.
// 1: ready; 0: a CUDA call failed; -1: not even one record fits.
constexpr int kZCIF6 = 4, kZCID6 = 2, kZCIF3 = 8, kZCID3 = 4;  // z chunk of the tile interpolation

template <typename T>
int spread_prepare(Plan& p) {
  constexpr int ZC6 = sizeof(T) == 4 ? kZC6F : kZC6D, ZC3 = sizeof(T) == 4 ? kZC3F : kZC3D;
  constexpr int ZCS = sizeof(T) == 4 ? kZCSF : kZCSD;
  constexpr int ZI6 = sizeof(T) == 4 ? kZCIF6 : kZCID6, ZI3 = sizeof(T) == 4 ? kZCIF3 : kZCID3;
  if (!(allow_smem(spread_kernel<T, 1, ZC6>) && allow_smem(spread_kernel<T, 0, ZC3>) &&
        allow_smem(spread_kernel<T, 2, ZC3>) && allow_smem(spread_kernel<T, 3, ZC3>) &&
        allow_smem(spread_kernel<T, 4, ZCS>) && allow_smem(interp_tile_kernel<T, 4, ZI6>) &&
        allow_smem(interp_tile_kernel<T, 0, ZI3>) && allow_smem(interp_stage_kernel<6>) &&
        allow_smem(interp_stage_kernel<3>)))
    return 0;
  int dev = 0, optin = 0;
  cudaFuncAttributes fa, fi;  // the spread modes declare the same static shared arrays; the tile
                              // interpolation adds its sums
  if (cudaGetDevice(&dev) != cudaSuccess ||
      cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev) != cudaSuccess ||
      cudaFuncGetAttributes(&fa, spread_kernel<T, 1, ZC6>) != cudaSuccess ||
      cudaFuncGetAttributes(&fi, interp_tile_kernel<T, 4, ZI6>) != cudaSuccess)
    return 0;
  const long rb = (long)p.g.rec_words * (long)sizeof(uint32_t);
  const long cap = ((long)optin - (long)std::max(fa.sharedSizeBytes, fi.sharedSizeBytes)) / rb;
  p.g.stage_cap = (int)std::min<long>(kStage, cap);
  // records built in shared memory by blocks of 128, 64 or 32 threads when that many fit in
  // 96 KB (two blocks per SM), else written directly
  if (!allow_smem(records_kernel<T, true>)) return 0;
  p.g.rec_threads = 0;
  for (int t : {128, 64, 32})
    if ((long)t * rb <= 96 * 1024) { p.g.rec_threads = t; break; }
  return p.g.stage_cap >= 1 ? 1 : -1;
}

template <typename T>
void launch_spread(const Plan& p, cudaStream_t s) {
  const unsigned blocks = (unsigned)(p.g.nbx * p.g.nby);
  constexpr int ZC6 = sizeof(T) == 4 ? kZC6F : kZC6D, ZC3 = sizeof(T) == 4 ? kZC3F : kZC3D;
  const size_t sm = spread_smem<T>(p);
  constexpr int ZCS = sizeof(T) == 4 ? kZCSF : kZCSD;
  T* grid = reinterpret_cast<T*>(p.grid);
  if (p.g.spectral_curl && p.g.kM.px == p.g.kD.px)  // equal m: the two supports coincide
    spread_kernel<T, 4, ZCS><<<blocks, kSpreadThreads, sm, s>>>(p.g, p.records, p.bin_start, p.sorted, p.zrange, grid);
  else if (p.g.spectral_curl)
    spread_kernel<T, 1, ZC6><<<blocks, kSpreadThreads, sm, s>>>(p.g, p.records, p.bin_start, p.sorted, p.zrange, grid);
  else if (p.g.torque_deriv && p.g.kM.px == p.g.kD.px)  // equal m: the two supports coincide
    spread_kernel<T, 3, ZC3><<<blocks, kSpreadThreads, sm, s>>>(p.g, p.records, p.bin_start, p.sorted, p.zrange, grid);
  else if (p.g.torque_deriv)
    spread_kernel<T, 2, ZC3><<<blocks, kSpreadThreads, sm, s>>>(p.g, p.records, p.bin_start, p.sorted, p.zrange, grid);
  else
    spread_kernel<T, 0, ZC3><<<blocks, kSpreadThreads, sm, s>>>(p.g, p.records, p.bin_start, p.sorted, p.zrange, grid);
}

// the tile-gather interpolation applies: forces only, or spectral-curl torques with coinciding
// supports; returns the fields it sums (0: not applicable)
int interp_tile_fields(const Geometry& g) {
  if (g.torque_deriv) return 0;
  if (g.spectral_curl) return g.kM.px == g.kD.px ? 6 : 0;
  return 3;
}

// the staged-grid interpolation applies (float plans; supports of at most kIsPX nodes; forces only
// or spectral-curl torques with coinciding supports); returns the fields it sums (0: not applicable)
int interp_stage_fields(const Geometry& g, int tsize) {
  if (tsize != 1 || g.pxc > kIsPX || g.lzc > kIsZT) return 0;
  return interp_tile_fields(g);
}

// the grid's real values as a rank-4 tensor (x, y, plane, field) with boxes of the staged layout:
// kIsSX columns x kIsRows rows x kIsGroups planes x the kernel's fields
bool encode_interp_tmap(Plan& p) {
  void* fn = nullptr;
  cudaDriverEntryPointQueryResult q;
  if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &fn, 12000, cudaEnableDefault, &q) != cudaSuccess ||
      q != cudaDriverEntryPointSuccess || fn == nullptr) {
    cudaGetLastError();
    return false;
  }
  auto encode = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(fn);
  const Geometry& g = p.g;
  const int nf = interp_stage_fields(g, 1);
  if (nf == 0 || g.nx < kIsSX) return false;
  const size_t rowb = (size_t)2 * g.pitch * sizeof(float);
  const cuuint64_t dims[4] = {(cuuint64_t)g.nx, (cuuint64_t)g.ny, (cuuint64_t)g.nz, (cuuint64_t)nf};
  const cuuint64_t strides[3] = {(cuuint64_t)rowb, (cuuint64_t)(rowb * g.ny), (cuuint64_t)(rowb * g.ny * g.nz)};
  const cuuint32_t box[4] = {(cuuint32_t)kIsSX, (cuuint32_t)kIsRows, (cuuint32_t)kIsGroups, (cuuint32_t)nf};
  const cuuint32_t estr[4] = {1, 1, 1, 1};
  CUtensorMap* map = reinterpret_cast<CUtensorMap*>(p.interp_tmap);
  return encode(map, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 4, p.grid, dims, strides, box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE,
                CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_NONE,
                CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

// tiles a support can overlap in x and y (a partial last tile can add one) and the partial-sum
// buffer of the tile-gather interpolation, in values of the transform precision
void interp_tile_slots(const Geometry& g, int& sxn, int& syn) {
  sxn = std::min(g.nbx, (g.kM.px - 1) / kTileX + 2 + ((g.nx % kTileX) ? 1 : 0));
  syn = std::min(g.nby, (g.kM.px - 1) / kTileY + 2 + ((g.ny % kTileY) ? 1 : 0));
}

size_t interp_tile_values(const Geometry& g, int64_t max_n) {
  const int nf = interp_tile_fields(g);
  if (nf == 0) return 0;
  int sxn, syn;
  interp_tile_slots(g, sxn, syn);
  return (size_t)sxn * syn * nf * (size_t)std::max<int64_t>(max_n, 1);
}

template <typename T>
void launch_interp(const Plan& p, int64_t n, double* U, double* W, cudaStream_t s) {
  if (n <= 0) return;
  const int threads = 256;
  const unsigned blocks = (unsigned)((n * 32 + threads - 1) / threads);
  const T* grid = reinterpret_cast<const T*>(p.grid);
  const T* wz = reinterpret_cast<const T*>(p.tab.wz);
  const int nf = interp_tile_fields(p.g);
  if constexpr (sizeof(T) == 4) {
    const int ns = interp_stage_fields(p.g, 1);
    if (p.interp_tile == 2 && ns > 0) {
      const unsigned bins = (unsigned)(p.g.nbx * p.g.nby);
      const int force_global = p.inject == 2 ? 1 : 0;  // test hook: every bin takes the global gather
      const CUtensorMap& map = *reinterpret_cast<const CUtensorMap*>(p.interp_tmap);
      if (ns == 6)
        interp_stage_kernel<6><<<bins, kIsThreads, interp_stage_smem(6), s>>>(
            map, p.interp_tma, p.g, p.records, p.bin_start, p.sorted, grid, wz, U, W, force_global, p.status);
      else
        interp_stage_kernel<3><<<bins, kIsThreads, interp_stage_smem(3), s>>>(
            map, p.interp_tma, p.g, p.records, p.bin_start, p.sorted, grid, wz, U, W, force_global, p.status);
      return;
    }
  }
  if (p.interp_tile == 1 && nf > 0 && p.ipart) {
    int sxn, syn;
    interp_tile_slots(p.g, sxn, syn);
    T* part = reinterpret_cast<T*>(p.ipart);
    const unsigned tiles = (unsigned)(p.g.nbx * p.g.nby);
    const size_t sm = spread_smem<T>(p);
    const unsigned fb = (unsigned)((n + 255) / 256);
    if (nf == 6) {
      constexpr int ZI = sizeof(T) == 4 ? kZCIF6 : kZCID6;
      interp_tile_kernel<T, 4, ZI><<<tiles, kSpreadThreads, sm, s>>>(p.g, p.records, p.bin_start, p.sorted, p.zrange,
                                                                     grid, wz, part, n, sxn, syn, p.status);
      interp_finish_kernel<T, 4><<<fb, 256, 0, s>>>(p.g, n, p.records, part, sxn, syn, U, W);
    } else {
      constexpr int ZI = sizeof(T) == 4 ? kZCIF3 : kZCID3;
      interp_tile_kernel<T, 0, ZI><<<tiles, kSpreadThreads, sm, s>>>(p.g, p.records, p.bin_start, p.sorted, p.zrange,
                                                                     grid, wz, part, n, sxn, syn, p.status);
      interp_finish_kernel<T, 0><<<fb, 256, 0, s>>>(p.g, n, p.records, part, sxn, syn, U, W);
    }
    return;
  }
  // lanes per x run: the narrowest group that holds a support row
  if (p.g.torque_deriv) {
    const bool fused = p.g.kM.px == p.g.kD.px;  // equal m: identical supports (alpha = m h / 2)
    if (p.g.pxc <= 6) {
      if (fused) interp_curl_kernel<T, 6, true><<<blocks, threads, 0, s>>>(p.g, n, p.records, grid, wz, p.sorted, U, W);
      else interp_curl_kernel<T, 6, false><<<blocks, threads, 0, s>>>(p.g, n, p.records, grid, wz, p.sorted, U, W);
    } else if (p.g.pxc <= 8) {
      if (fused) interp_curl_kernel<T, 8, true><<<blocks, threads, 0, s>>>(p.g, n, p.records, grid, wz, p.sorted, U, W);
      else interp_curl_kernel<T, 8, false><<<blocks, threads, 0, s>>>(p.g, n, p.records, grid, wz, p.sorted, U, W);
    } else {
      if (fused) interp_curl_kernel<T, 16, true><<<blocks, threads, 0, s>>>(p.g, n, p.records, grid, wz, p.sorted, U, W);
      else interp_curl_kernel<T, 16, false><<<blocks, threads, 0, s>>>(p.g, n, p.records, grid, wz, p.sorted, U, W);
    }
    return;
  }
  if (p.g.spectral_curl && p.g.kM.px == p.g.kD.px) {  // equal m: one walk for U and Omega
    if (p.g.pxc <= 6)
      interp_pair_kernel<T, 6><<<blocks, threads, 0, s>>>(p.g, n, p.records, grid, wz, p.sorted, U, W);
    else if (p.g.pxc <= 8)
      interp_pair_kernel<T, 8><<<blocks, threads, 0, s>>>(p.g, n, p.records, grid, wz, p.sorted, U, W);
    else
      interp_pair_kernel<T, 16><<<blocks, threads, 0, s>>>(p.g, n, p.records, grid, wz, p.sorted, U, W);
    return;
  }
  if (p.g.pxc <= 6)
    interp_kernel<T, 6><<<blocks, threads, 0, s>>>(p.g, n, p.records, grid, wz, p.sorted, U, W);
  else if (p.g.pxc <= 8)
    interp_kernel<T, 8><<<blocks, threads, 0, s>>>(p.g, n, p.records, grid, wz, p.sorted, U, W);
  else
    interp_kernel<T, 16><<<blocks, threads, 0, s>>>(p.g, n, p.records, grid, wz, p.sorted, U, W);
}

template void launch_records<float>(const Plan&, int64_t, const double*, const double*, const double*, cudaStream_t);
template void launch_records<double>(const Plan&, int64_t, const double*, const double*, const double*, cudaStream_t);
template void launch_spread<float>(const Plan&, cudaStream_t);
template int spread_prepare<float>(Plan&);
template int spread_prepare<double>(Plan&);
template void launch_spread<double>(const Plan&, cudaStream_t);
template void launch_interp<float>(const Plan&, int64_t, double*, double*, cudaStream_t);
template void launch_interp<double>(const Plan&, int64_t, double*, double*, cudaStream_t);

}  // namespace dps
