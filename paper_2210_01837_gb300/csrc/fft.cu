// In-house xy FFTs of the Chebyshev planes (steps 2 and 7 of Sec. III.D, xy part).
//
// Forward: f_hat(k) = sum_x f(x) exp(-i k.x) (unnormalised).  Inverse: sum_k f_hat(k) exp(+i k.x);
// the 1/(Nx Ny) factor is applied by the per-k solver when it writes its outputs.
//
// Layout of one field/plane: ny rows; each row holds nx reals in real space and nx/2+1 complex
// values (pitch >= nx/2+1 complex) in x-Fourier space, in place.
//   * row pass:    a unit is two real rows packed as one complex sequence (z = r0 + i r1), whose
//                  transform is then split into the two half spectra; inverse likewise.
//   * column pass: a unit is `cw` adjacent x-wavenumber columns of one plane, transformed along y.
// Both passes run persistent blocks (as many as fit on the GPU) that walk the units of the live
// planes, in one of two variants.  Shared-memory-staged: a block stages a unit in shared memory
// with cp.async; the first stage reads the staged values directly, after which the staging buffer
// takes the next unit's copies while the later stages alternate between two padded work buffers,
// so HBM traffic overlaps the butterflies and each unit crosses shared memory 2 S + 2 times for S
// stages.  Register-staged: one butterfly per thread and stage, updated in place in one shared
// buffer, the first stage reading HBM and the last writing it directly (described further below);
// for the column pass also with a second buffer that receives the next unit, by cp.async or by
// TMA box loads on an mbarrier.
// The plan picks the variant per pass (default rule at fft_smem_ok, or autotuned / set by hand).
// Each 1D transform is a self-sorting (Stockham) mixed-radix FFT in shared memory written from the
// textbook formulation: stage s with radix R and span Ns multiplies input j + r n/R by
// W_{Ns R}^{(j mod Ns) r}, applies an R-point DFT, and stores to (j / Ns) Ns R + (j mod Ns) + r Ns.
// Radices 16, 12 (as 4 x 4 and 4 x 3), 8, 4, 2 (hand-written butterflies) and 3, 5, 7 (direct DFT
// with exact constants).  Twiddles W_n^t = exp(-2 pi i t/n) come from a table built in double
// precision on the host; the register-staged column passes read per-stage rows W_{Ns R}^{k r}
// instead (one contiguous row per butterfly).
#include <cuda.h>
#include <cudaTypedefs.h>

#include <algorithm>

#include "dps_internal.cuh"
#include "fft_pair.h"

namespace dps {

namespace {

// cos(2 pi m / R) and sin(2 pi m / R) as literals in the transform's own precision (no conversions
// in the butterflies: on this GPU a float<->double conversion occupies the scarce FP64 pipe).  The
// butterfly loops are fully unrolled, so m is a compile-time constant and the switches fold away.
template <typename T, int R>
__device__ __forceinline__ T root_cos(int m) {
  if (R == 3) return m == 0 ? (T)1.0 : (T)-0.5;
  if (R == 5) {
    switch (m) {
      case 0: return (T)1.0;
      case 1: case 4: return (T)0.30901699437494742;
      default: return (T)-0.80901699437494742;
    }
  }
  switch (m) {
    case 0: return (T)1.0;
    case 1: case 6: return (T)0.62348980185873353;
    case 2: case 5: return (T)-0.22252093395631440;
    default: return (T)-0.90096886790241913;
  }
}

template <typename T, int R>
__device__ __forceinline__ T root_sin(int m) {
  if (R == 3) return m == 0 ? (T)0.0 : (m == 1 ? (T)0.86602540378443865 : (T)-0.86602540378443865);
  if (R == 5) {
    switch (m) {
      case 0: return (T)0.0;
      case 1: return (T)0.95105651629515357;
      case 2: return (T)0.58778525229247314;
      case 3: return (T)-0.58778525229247314;
      default: return (T)-0.95105651629515357;
    }
  }
  switch (m) {
    case 0: return (T)0.0;
    case 1: return (T)0.78183148246802981;
    case 2: return (T)0.97492791218182361;
    case 3: return (T)0.43388373911755812;
    case 4: return (T)-0.43388373911755812;
    case 5: return (T)-0.97492791218182361;
    default: return (T)-0.78183148246802981;
  }
}

template <typename T, int DIR>
__device__ __forceinline__ cplx<T> rot_quarter(cplx<T> a) {
  // multiply by -i (forward) or +i (inverse)
  return DIR < 0 ? mk<T>(a.y, -a.x) : mk<T>(-a.y, a.x);
}

template <typename T, int R, int DIR> struct Dft;

template <typename T, int DIR> struct Dft<T, 2, DIR> {
  static __device__ __forceinline__ void run(cplx<T>* v) {
    const cplx<T> a = v[0], b = v[1];
    v[0] = a + b;
    v[1] = a - b;
  }
};

template <typename T, int DIR> struct Dft<T, 4, DIR> {
  static __device__ __forceinline__ void run(cplx<T>* v) {
    const cplx<T> t0 = v[0] + v[2], t1 = v[0] - v[2], t2 = v[1] + v[3];
    const cplx<T> t3 = rot_quarter<T, DIR>(v[1] - v[3]);
    v[0] = t0 + t2;
    v[2] = t0 - t2;
    v[1] = t1 + t3;
    v[3] = t1 - t3;
  }
};

template <typename T, int DIR> struct Dft<T, 8, DIR> {
  static __device__ __forceinline__ void run(cplx<T>* v) {
    cplx<T> e[4] = {v[0], v[2], v[4], v[6]};
    cplx<T> o[4] = {v[1], v[3], v[5], v[7]};
    Dft<T, 4, DIR>::run(e);
    Dft<T, 4, DIR>::run(o);
    const T s = (T)0.70710678118654752440;
    // W8^k, k = 0..3, for the transform direction
    const cplx<T> w1 = mk<T>(s, (T)DIR * s);
    const cplx<T> w3 = mk<T>(-s, (T)DIR * s);
    const cplx<T> o1 = o[1] * w1;
    const cplx<T> o2 = rot_quarter<T, DIR>(o[2]);
    const cplx<T> o3 = o[3] * w3;
    v[0] = e[0] + o[0];
    v[4] = e[0] - o[0];
    v[1] = e[1] + o1;
    v[5] = e[1] - o1;
    v[2] = e[2] + o2;
    v[6] = e[2] - o2;
    v[3] = e[3] + o3;
    v[7] = e[3] - o3;
  }
};

// 16-point DFT as 4 x 4: x[4a + b] -> X[c + 4d];  inner DFT4 over a, twiddle W16^(b c), outer DFT4 over b
template <typename T, int DIR> struct Dft<T, 16, DIR> {
  static __device__ __forceinline__ void run(cplx<T>* v) {
    // cos(2 pi m / 16), m = 0..3, and the matching sines
    const T c1 = (T)0.92387953251128676, s1 = (T)0.38268343236508977, h = (T)0.70710678118654752;
    cplx<T> t[4][4];
#pragma unroll
    for (int b = 0; b < 4; ++b) {
      cplx<T> w[4] = {v[b], v[4 + b], v[8 + b], v[12 + b]};
      Dft<T, 4, DIR>::run(w);
#pragma unroll
      for (int c = 0; c < 4; ++c) t[b][c] = w[c];
    }
    // twiddles W16^(b c) for b, c in 1..3 (sign of the imaginary part follows the direction)
    const T sg = (T)DIR;
    t[1][1] = t[1][1] * mk<T>(c1, sg * s1);
    t[1][2] = t[1][2] * mk<T>(h, sg * h);
    t[1][3] = t[1][3] * mk<T>(s1, sg * c1);
    t[2][1] = t[2][1] * mk<T>(h, sg * h);
    t[2][2] = rot_quarter<T, DIR>(t[2][2]);
    t[2][3] = t[2][3] * mk<T>(-h, sg * h);
    t[3][1] = t[3][1] * mk<T>(s1, sg * c1);
    t[3][2] = t[3][2] * mk<T>(-h, sg * h);
    t[3][3] = t[3][3] * mk<T>(-c1, -sg * s1);
#pragma unroll
    for (int c = 0; c < 4; ++c) {
      cplx<T> w[4] = {t[0][c], t[1][c], t[2][c], t[3][c]};
      Dft<T, 4, DIR>::run(w);
#pragma unroll
      for (int d = 0; d < 4; ++d) v[c + 4 * d] = w[d];
    }
  }
};

template <typename T, int R, int DIR>
__device__ __forceinline__ void dft_direct(cplx<T>* v) {
  cplx<T> out[R];
#pragma unroll
  for (int k = 0; k < R; ++k) {
    cplx<T> acc = v[0];
#pragma unroll
    for (int r = 1; r < R; ++r) {
      const int m = (r * k) % R;
      const cplx<T> w = mk<T>(root_cos<T, R>(m), DIR > 0 ? root_sin<T, R>(m) : -root_sin<T, R>(m));
      acc = acc + v[r] * w;
    }
    out[k] = acc;
  }
#pragma unroll
  for (int k = 0; k < R; ++k) v[k] = out[k];
}

template <typename T, int DIR> struct Dft<T, 3, DIR> {
  static __device__ __forceinline__ void run(cplx<T>* v) { dft_direct<T, 3, DIR>(v); }
};
template <typename T, int DIR> struct Dft<T, 5, DIR> {
  static __device__ __forceinline__ void run(cplx<T>* v) { dft_direct<T, 5, DIR>(v); }
};
template <typename T, int DIR> struct Dft<T, 7, DIR> {
  static __device__ __forceinline__ void run(cplx<T>* v) { dft_direct<T, 7, DIR>(v); }
};

// 12-point DFT as 4 x 3: x[3 a + b] -> X[c + 4 d]; inner DFT4 over a, twiddle W12^(b c), outer DFT3 over b
template <typename T, int DIR> struct Dft<T, 12, DIR> {
  static __device__ __forceinline__ void run(cplx<T>* v) {
    const T h = (T)0.5, s3 = (T)0.86602540378443865, sg = (T)DIR;  // cos/sin of 30 and 60 degrees
    cplx<T> y[3][4];
#pragma unroll
    for (int b = 0; b < 3; ++b) {
      cplx<T> w[4] = {v[b], v[3 + b], v[6 + b], v[9 + b]};
      Dft<T, 4, DIR>::run(w);
#pragma unroll
      for (int c = 0; c < 4; ++c) y[b][c] = w[c];
    }
    // W12^m = (cos(2 pi m / 12), DIR sin(2 pi m / 12)) for m = b c
    y[1][1] = y[1][1] * mk<T>(s3, sg * h);
    y[1][2] = y[1][2] * mk<T>(h, sg * s3);
    y[1][3] = rot_quarter<T, DIR>(y[1][3]);
    y[2][1] = y[2][1] * mk<T>(h, sg * s3);
    y[2][2] = y[2][2] * mk<T>(-h, sg * s3);
    y[2][3] = mk<T>(-y[2][3].x, -y[2][3].y);
#pragma unroll
    for (int c = 0; c < 4; ++c) {
      cplx<T> w[3] = {y[0][c], y[1][c], y[2][c]};
      Dft<T, 3, DIR>::run(w);
#pragma unroll
      for (int d = 0; d < 3; ++d) v[c + 4 * d] = w[d];
    }
  }
};

// Shared-memory index with one pad element per 16: breaks the power-of-two strides of the
// Stockham writes across bank groups.
__device__ __forceinline__ int pad16(int i) { return i + (i >> 4); }

// A transform of n points over 2^lbatch interleaved sequences runs on about n 2^lbatch / kFftPer
// threads (whole warps), so a radix-R stage gives each thread about kFftPer / R butterflies.
constexpr int kFftPer = 12;

// First Stockham stage (span 1, no twiddles): butterfly (jj, b) reads elements jj + r n/R of
// sequence b through `in(flat index)` and writes X to buf[(jj R + r) 2^lbatch + b] (padded).
template <typename T, int R, int DIR, class In>
__device__ __forceinline__ void stage_first(cplx<T>* __restrict__ buf, int n, int lbatch, const In& in) {
  const int nr = n / R;
  const int total = nr << lbatch;
  const int bmask = (1 << lbatch) - 1;
  for (int t = threadIdx.x; t < total; t += blockDim.x) {
    const int b = t & bmask, jj = t >> lbatch;
    cplx<T> v[R];
#pragma unroll
    for (int r = 0; r < R; ++r) v[r] = in(((jj + r * nr) << lbatch) + b);
    Dft<T, R, DIR>::run(v);
#pragma unroll
    for (int r = 0; r < R; ++r) buf[pad16(((jj * R + r) << lbatch) + b)] = v[r];
  }
}

// Later stage (span Ns), out of place: stage s multiplies input j + r n/R by W_{Ns R}^{(j mod Ns) r},
// applies an R-point DFT and stores to (j / Ns) Ns R + (j mod Ns) + r Ns; the division by Ns is a
// multiply-high with a per-stage magic number (exact below 2^20).
template <typename T, int R, int DIR>
__device__ __forceinline__ void stage(const cplx<T>* __restrict__ in, cplx<T>* __restrict__ out, int n, int Ns,
                                      unsigned long long magic, int lbatch, const cplx<T>* __restrict__ tw) {
  const int nr = n / R;
  const int total = nr << lbatch;
  const int bmask = (1 << lbatch) - 1;
  const int tstep = n / (Ns * R);
  for (int t = threadIdx.x; t < total; t += blockDim.x) {
    const int b = t & bmask, jj = t >> lbatch;
    const int q = (int)(((unsigned long long)jj * magic) >> 40);
    const int k = jj - q * Ns;
    cplx<T> v[R];
#pragma unroll
    for (int r = 0; r < R; ++r) v[r] = in[pad16(((jj + r * nr) << lbatch) + b)];
#pragma unroll
    for (int r = 1; r < R; ++r) {
      cplx<T> w = tw[k * r * tstep];
      if (DIR > 0) w.y = -w.y;
      v[r] = v[r] * w;
    }
    Dft<T, R, DIR>::run(v);
    const int base = q * Ns * R + k;
#pragma unroll
    for (int r = 0; r < R; ++r) out[pad16(((base + r * Ns) << lbatch) + b)] = v[r];
  }
}

template <typename T, int DIR, class In>
__device__ __forceinline__ void fft_first(cplx<T>* buf, const FftPlan& fp, int lbatch, const In& in) {
  switch (fp.radix[0]) {
    case 16: stage_first<T, 16, DIR>(buf, fp.n, lbatch, in); break;
    case 12: stage_first<T, 12, DIR>(buf, fp.n, lbatch, in); break;
    case 8: stage_first<T, 8, DIR>(buf, fp.n, lbatch, in); break;
    case 4: stage_first<T, 4, DIR>(buf, fp.n, lbatch, in); break;
    case 2: stage_first<T, 2, DIR>(buf, fp.n, lbatch, in); break;
    case 3: stage_first<T, 3, DIR>(buf, fp.n, lbatch, in); break;
    case 5: stage_first<T, 5, DIR>(buf, fp.n, lbatch, in); break;
    default: stage_first<T, 7, DIR>(buf, fp.n, lbatch, in); break;
  }
}

// stages 1 .. nstages-1, alternating between the two work buffers (each ends with a block
// barrier); returns the buffer that holds the transform
template <typename T, int DIR>
__device__ cplx<T>* fft_rest(cplx<T>* b0, cplx<T>* b1, const FftPlan& fp, int lbatch, const cplx<T>* tw) {
  int Ns = fp.radix[0];
  cplx<T>* in = b0;
  cplx<T>* out = b1;
  for (int s = 1; s < fp.nstages; ++s) {
    const int R = fp.radix[s];
    const unsigned long long mg = fp.magic[s];
    switch (R) {
      case 16: stage<T, 16, DIR>(in, out, fp.n, Ns, mg, lbatch, tw); break;
      case 12: stage<T, 12, DIR>(in, out, fp.n, Ns, mg, lbatch, tw); break;
      case 8: stage<T, 8, DIR>(in, out, fp.n, Ns, mg, lbatch, tw); break;
      case 4: stage<T, 4, DIR>(in, out, fp.n, Ns, mg, lbatch, tw); break;
      case 2: stage<T, 2, DIR>(in, out, fp.n, Ns, mg, lbatch, tw); break;
      case 3: stage<T, 3, DIR>(in, out, fp.n, Ns, mg, lbatch, tw); break;
      case 5: stage<T, 5, DIR>(in, out, fp.n, Ns, mg, lbatch, tw); break;
      default: stage<T, 7, DIR>(in, out, fp.n, Ns, mg, lbatch, tw); break;
    }
    __syncthreads();
    Ns *= R;
    cplx<T>* t = in;
    in = out;
    out = t;
  }
  return in;
}

// `bytes` (a multiple of 4) from a 16-byte aligned global address to a 16-byte aligned shared one
__device__ __forceinline__ void async_bytes(void* s, const void* g, int bytes) {
  const int n16 = bytes >> 4;
  char* sc = reinterpret_cast<char*>(s);
  const char* gc = reinterpret_cast<const char*>(g);
  for (int i = threadIdx.x; i < n16; i += blockDim.x) cp_async16(sc + 16 * i, gc + 16 * i);
  for (int i = 4 * n16 + threadIdx.x; i < (bytes >> 2); i += blockDim.x) cp_async4(sc + 4 * i, gc + 4 * i);
}

// Work units of the persistent transforms: (field, live plane, unit within the plane), unit fastest.
struct UnitMap {
  int clo, nlive, per_plane;
  long long total;
  __device__ UnitMap(const Geometry& g, const int* zrange, int per) {
    clo = zrange[0];
    nlive = max(0, zrange[1] - clo + 1);
    per_plane = per;
    total = (long long)g.nfields * nlive * per;
  }
  __device__ void at(long long u, int& f, int& c, int& j) const {
    j = (int)(u % per_plane);
    const long long r = u / per_plane;
    c = clo + (int)(r % nlive);
    f = (int)(r / nlive);
  }
};

// real rows rounded up so that the second staged row stays 16-byte aligned
__host__ __device__ __forceinline__ int staged_len(int n) { return (n + 3) & ~3; }

// Row pass, forward: a unit is two real rows y0 = 2j, y1 = 2j + 1, packed as z = r0 + i r1.
template <typename T>
__global__ void __launch_bounds__(512, 1) row_r2c_kernel(Geometry g, FftPlan fp, const cplx<T>* __restrict__ tw,
                                                         T* __restrict__ grid, const int* __restrict__ zrange) {
  extern __shared__ __align__(16) unsigned char smraw[];
  const int nx = g.nx, nxr = staged_len(nx);
  T* raw = reinterpret_cast<T*>(smraw);  // [2][nxr] staged rows
  cplx<T>* b0 = reinterpret_cast<cplx<T>*>(raw + 2 * nxr);
  cplx<T>* b1 = b0 + pad16(nx) + 1;
  cplx<T>* stw = b1 + pad16(nx) + 1;  // twiddle table, staged once per (persistent) block
  for (int i = threadIdx.x; i < nx; i += blockDim.x) stw[i] = tw[i];
  const UnitMap um(g, zrange, (g.ny + 1) / 2);
  const size_t rowlen = (size_t)2 * g.pitch;
  auto row0_of = [&](long long u, bool& has1) {
    int f, c, j;
    um.at(u, f, c, j);
    has1 = 2 * j + 1 < g.ny;
    return grid + ((size_t)(f * g.nz + c) * g.ny + 2 * j) * rowlen;
  };
  auto issue = [&](long long u) {
    bool has1;
    const T* r0 = row0_of(u, has1);
    async_bytes(raw, r0, nx * (int)sizeof(T));
    if (has1) async_bytes(raw + nxr, r0 + rowlen, nx * (int)sizeof(T));
    cp_commit();
  };
  long long u = blockIdx.x;
  if (u < um.total) issue(u);
  for (; u < um.total; u += gridDim.x) {
    bool has1;
    T* row0 = row0_of(u, has1);
    cp_wait_all();
    __syncthreads();  // staged rows visible; the previous unit's epilogue is done with buf
    fft_first<T, -1>(b0, fp, 0, [&](int e) { return mk<T>(raw[e], has1 ? raw[nxr + e] : (T)0); });
    __syncthreads();  // staging buffer consumed
    if (u + gridDim.x < um.total) issue(u + gridDim.x);
    const cplx<T>* buf = fft_rest<T, -1>(b0, b1, fp, 0, stw);
    cplx<T>* c0 = reinterpret_cast<cplx<T>*>(row0);
    cplx<T>* c1 = reinterpret_cast<cplx<T>*>(row0 + rowlen);
    const T half = (T)0.5;
    for (int k = threadIdx.x; k <= nx / 2; k += blockDim.x) {
      const cplx<T> zk = buf[pad16(k)];
      const cplx<T> zm = conjg(buf[pad16(k == 0 ? 0 : nx - k)]);
      c0[k] = scl(zk + zm, half);
      if (has1) {
        const cplx<T> d = zk - zm;  // (zk - conj z_{-k}) / (2i)
        c1[k] = mk<T>(half * d.y, -half * d.x);
      }
    }
  }
}

// Row pass, inverse: two half spectra -> z with z_k = X0_k + i X1_k (Hermitian extension), one FFT.
template <typename T>
__global__ void __launch_bounds__(512, 1) row_c2r_kernel(Geometry g, FftPlan fp, const cplx<T>* __restrict__ tw,
                                                         T* __restrict__ grid, const int* __restrict__ zrange) {
  extern __shared__ __align__(16) unsigned char smraw[];
  const int nx = g.nx, nh = nx / 2 + 1, nhr = (nh + 1) & ~1;
  cplx<T>* raw = reinterpret_cast<cplx<T>*>(smraw);  // [2][nhr] staged half spectra
  cplx<T>* b0 = raw + 2 * nhr;
  cplx<T>* b1 = b0 + pad16(nx) + 1;
  cplx<T>* stw = b1 + pad16(nx) + 1;  // twiddle table, staged once per (persistent) block
  for (int i = threadIdx.x; i < nx; i += blockDim.x) stw[i] = tw[i];
  const UnitMap um(g, zrange, (g.ny + 1) / 2);
  const size_t rowlen = (size_t)2 * g.pitch;
  auto row0_of = [&](long long u, bool& has1) {
    int f, c, j;
    um.at(u, f, c, j);
    has1 = 2 * j + 1 < g.ny;
    return grid + ((size_t)(f * g.nz + c) * g.ny + 2 * j) * rowlen;
  };
  auto issue = [&](long long u) {
    bool has1;
    const T* r0 = row0_of(u, has1);
    async_bytes(raw, r0, nh * (int)sizeof(cplx<T>));
    if (has1) async_bytes(raw + nhr, r0 + rowlen, nh * (int)sizeof(cplx<T>));
    cp_commit();
  };
  long long u = blockIdx.x;
  if (u < um.total) issue(u);
  for (; u < um.total; u += gridDim.x) {
    bool has1;
    T* row0 = row0_of(u, has1);
    T* row1 = row0 + rowlen;
    cp_wait_all();
    __syncthreads();
    fft_first<T, +1>(b0, fp, 0, [&](int e) {
      const bool lo = e <= nx / 2;
      const int k = lo ? e : nx - e;
      const cplx<T> x0 = raw[k];
      const cplx<T> x1 = has1 ? raw[nhr + k] : mk<T>((T)0, (T)0);
      return lo ? x0 + mul_i(x1) : conjg(x0) + mul_i(conjg(x1));
    });
    __syncthreads();
    if (u + gridDim.x < um.total) issue(u + gridDim.x);
    const cplx<T>* buf = fft_rest<T, +1>(b0, b1, fp, 0, stw);
    for (int a = threadIdx.x; a < nx; a += blockDim.x) {
      const cplx<T> v = buf[pad16(a)];
      row0[a] = v.x;
      if (has1) row1[a] = v.y;
    }
  }
}

// Column pass: a unit is cw adjacent x-wavenumber columns [kx0, kx0 + cw) of one plane, along y.
template <typename T, int DIR>
__global__ void __launch_bounds__(512, 1) col_kernel(Geometry g, FftPlan fp, const cplx<T>* __restrict__ tw,
                                                     cplx<T>* __restrict__ grid, const int* __restrict__ zrange,
                                                     int lcw, int kxs, int kxe) {
  extern __shared__ __align__(16) unsigned char smraw[];
  const int cw = 1 << lcw;
  const int tot = g.ny << lcw;
  cplx<T>* raw = reinterpret_cast<cplx<T>*>(smraw);  // [ny][cw] staged columns
  cplx<T>* b0 = raw + tot;
  cplx<T>* b1 = b0 + pad16(tot) + 1;
  cplx<T>* stw = b1 + pad16(tot) + 1;  // twiddle table, staged once per (persistent) block
  for (int i = threadIdx.x; i < g.ny; i += blockDim.x) stw[i] = tw[i];
  const UnitMap um(g, zrange, (kxe - kxs + cw - 1) >> lcw);
  auto base_of = [&](long long u, int& ncols) {
    int f, c, j;
    um.at(u, f, c, j);
    const int kx0 = kxs + (j << lcw);
    ncols = min(cw, kxe - kx0);
    return grid + (size_t)(f * g.nz + c) * g.ny * g.pitch + kx0;
  };
  auto issue = [&](long long u) {
    int ncols;
    const cplx<T>* base = base_of(u, ncols);
    const bool wide = ncols == cw && (cw * sizeof(cplx<T>)) % 16 == 0 &&
                      (reinterpret_cast<size_t>(base) & 15) == 0;
    if (wide) {
      const int per = (cw * (int)sizeof(cplx<T>)) >> 4;  // 16-byte pieces per row
      for (int t = threadIdx.x; t < g.ny * per; t += blockDim.x) {
        const int y = t / per, q = t - y * per;
        cp_async16(reinterpret_cast<char*>(raw + (y << lcw)) + 16 * q,
                   reinterpret_cast<const char*>(base + (size_t)y * g.pitch) + 16 * q);
      }
    } else {
      for (int t = threadIdx.x; t < tot; t += blockDim.x) {
        const int y = t >> lcw, b = t & (cw - 1);
        if (b < ncols) async_elem(raw + t, base + (size_t)y * g.pitch + b);
      }
    }
    cp_commit();
  };
  long long u = blockIdx.x;
  if (u < um.total) issue(u);
  for (; u < um.total; u += gridDim.x) {
    int ncols;
    cplx<T>* base = base_of(u, ncols);
    cp_wait_all();
    __syncthreads();
    fft_first<T, DIR>(b0, fp, lcw, [&](int t) { return ((t & (cw - 1)) < ncols) ? raw[t] : mk<T>((T)0, (T)0); });
    __syncthreads();
    if (u + gridDim.x < um.total) issue(u + gridDim.x);
    const cplx<T>* buf = fft_rest<T, DIR>(b0, b1, fp, lcw, stw);
    for (int t = threadIdx.x; t < tot; t += blockDim.x) {
      const int y = t >> lcw, b = t & (cw - 1);
      if (b < ncols) base[(size_t)y * g.pitch + b] = buf[pad16(t)];
    }
  }
}

// ---- register-staged variant ----
// Each thread owns at most one butterfly per stage (the block has at least as many threads as the
// stage with the most butterflies): it reads the butterfly's R inputs, applies the twiddles and the
// R-point DFT in registers and, after a block barrier, writes the R outputs back in place, so the
// block needs one unit-sized shared buffer instead of a staging buffer and two work buffers.  The
// first stage reads HBM directly and (column pass and inverse row pass) the last stage writes HBM
// directly, so a unit crosses shared memory 2 (S - 1) times for S stages and the resident blocks
// (several per SM) hide each other's memory latency.

// One stage (radix R, span Ns) over 2^lb interleaved sequences: butterfly t = (jj, b) reads
// element jj + r n/R of sequence b through src(element, b), multiplies input r by
// W_{Ns R}^{(jj mod Ns) r} (stages after the first), and stores X_r as element
// (jj / Ns) Ns R + (jj mod Ns) + r Ns through dst(element, b, X_r).  With `barrier` every thread
// has read its inputs before any thread writes (in-place update).
// The in-place shared buffer of a register-staged transform: value i at p[i + PW (i >> 4)].
template <int PW, int SH = 4>
__device__ __forceinline__ int padw(int i) { return i + PW * (i >> SH); }

// a shared transform buffer padded with PW values after every 2^SH
template <typename T, int PW, int SH = 4>
struct ShBuf {
  cplx<T>* p;
  int lb;
};

// R values e0 + r es (r < R) of sequence b: through the accessor, or, for the shared buffer, from
// one padded base plus a padded stride when the flat stride es 2^lb is a multiple of 16 (then the
// padding is linear in r), which saves the per-value index arithmetic.
template <typename T, int R, class Src>
__device__ __forceinline__ void load_all(cplx<T>* v, const Src& src, int e0, int es, int b) {
#pragma unroll
  for (int r = 0; r < R; ++r) v[r] = src(e0 + r * es, b);
}
template <typename T, int R, int PW, int SH>
__device__ __forceinline__ void load_all(cplx<T>* v, const ShBuf<T, PW, SH>& sb, int e0, int es, int b) {
  const int i0 = (e0 << sb.lb) + b, S = es << sb.lb;
  if ((S & ((1 << SH) - 1)) == 0) {
    const int p0 = padw<PW, SH>(i0), Sp = S + PW * (S >> SH);
#pragma unroll
    for (int r = 0; r < R; ++r) v[r] = sb.p[p0 + r * Sp];
  } else {
#pragma unroll
    for (int r = 0; r < R; ++r) v[r] = sb.p[padw<PW, SH>(i0 + r * S)];
  }
}
template <typename T, int R, class Dst>
__device__ __forceinline__ void store_all(const cplx<T>* v, const Dst& dst, int e0, int es, int b) {
#pragma unroll
  for (int r = 0; r < R; ++r) dst(e0 + r * es, b, v[r]);
}
template <typename T, int R, int PW, int SH>
__device__ __forceinline__ void store_all(const cplx<T>* v, const ShBuf<T, PW, SH>& sb, int e0, int es, int b) {
  const int i0 = (e0 << sb.lb) + b, S = es << sb.lb;
  if ((S & ((1 << SH) - 1)) == 0) {
    const int p0 = padw<PW, SH>(i0), Sp = S + PW * (S >> SH);
#pragma unroll
    for (int r = 0; r < R; ++r) sb.p[p0 + r * Sp] = v[r];
  } else {
#pragma unroll
    for (int r = 0; r < R; ++r) sb.p[padw<PW, SH>(i0 + r * S)] = v[r];
  }
}

// v[r] *= row[r] (conjugated for the inverse), r = 1 .. R-1, row = one row of a stage-twiddle
// table (row[0] = 1); float rows of even R are 16-byte aligned and load two twiddles at a time.
template <typename T, int R, int DIR>
__device__ __forceinline__ void apply_twiddles(cplx<T>* v, const cplx<T>* __restrict__ row) {
  if (sizeof(T) == 4 && R % 2 == 0) {
#pragma unroll
    for (int r = 0; r < R; r += 2) {
      const float4 q = *reinterpret_cast<const float4*>(row + r);
      cplx<T> w1 = mk<T>((T)q.z, (T)q.w);
      if (DIR > 0) w1.y = -w1.y;
      if (r > 0) {
        cplx<T> w0 = mk<T>((T)q.x, (T)q.y);
        if (DIR > 0) w0.y = -w0.y;
        v[r] = v[r] * w0;
      }
      v[r + 1] = v[r + 1] * w1;
    }
  } else {
#pragma unroll
    for (int r = 1; r < R; ++r) {
      cplx<T> w = row[r];
      if (DIR > 0) w.y = -w.y;
      v[r] = v[r] * w;
    }
  }
}

// tw: with ST the stage-twiddle table of this transform (FftPlan::toff), else the length-n table
template <typename T, int R, int DIR, bool ST, class Src, class Dst>
__device__ __forceinline__ void reg_stage(const FftPlan& fp, int s, int Ns, int lb, const cplx<T>* __restrict__ tw,
                                          const Src& src, const Dst& dst, bool barrier) {
  const int n = fp.n, nr = n / R, total = nr << lb;
  const int t = threadIdx.x;
  const bool act = t < total;
  const int b = t & ((1 << lb) - 1), jj = t >> lb;
  cplx<T> v[R];  // initialised: an array left undefined on the idle threads' path is not kept in registers
#pragma unroll
  for (int r = 0; r < R; ++r) v[r] = mk<T>((T)0, (T)0);
  int ob = jj * R;
  if (act) {
    load_all<T, R>(v, src, jj, nr, b);
    if (s > 0) {
      const int q = (int)(((unsigned long long)jj * fp.magic[s]) >> 40);
      const int k = jj - q * Ns;
      if (ST) {
        apply_twiddles<T, R, DIR>(v, tw + fp.toff[s] + k * R);  // row k of the stage's W_{Ns R}^{k r}
      } else {
        const int kt = k * (n / (Ns * R));  // W_{Ns R}^{k r} = W_n^{kt r}
#pragma unroll
        for (int r = 1; r < R; ++r) {
          cplx<T> w = tw[kt * r];
          if (DIR > 0) w.y = -w.y;
          v[r] = v[r] * w;
        }
      }
      ob = q * Ns * R + k;
    }
    Dft<T, R, DIR>::run(v);
  }
  if (barrier) __syncthreads();
  if (act) store_all<T, R>(v, dst, ob, Ns, b);
}

template <typename T, int DIR, bool ST, class Src, class Dst>
__device__ __forceinline__ void reg_stage_any(const FftPlan& fp, int s, int Ns, int lb, const cplx<T>* tw,
                                              const Src& src, const Dst& dst, bool barrier) {
  switch (fp.radix[s]) {
    case 16: reg_stage<T, 16, DIR, ST>(fp, s, Ns, lb, tw, src, dst, barrier); break;
    case 12: reg_stage<T, 12, DIR, ST>(fp, s, Ns, lb, tw, src, dst, barrier); break;
    case 8: reg_stage<T, 8, DIR, ST>(fp, s, Ns, lb, tw, src, dst, barrier); break;
    case 4: reg_stage<T, 4, DIR, ST>(fp, s, Ns, lb, tw, src, dst, barrier); break;
    case 2: reg_stage<T, 2, DIR, ST>(fp, s, Ns, lb, tw, src, dst, barrier); break;
    case 3: reg_stage<T, 3, DIR, ST>(fp, s, Ns, lb, tw, src, dst, barrier); break;
    case 5: reg_stage<T, 5, DIR, ST>(fp, s, Ns, lb, tw, src, dst, barrier); break;
    default: reg_stage<T, 7, DIR, ST>(fp, s, Ns, lb, tw, src, dst, barrier); break;
  }
}

// A whole transform: src (HBM) -> stages in the shared buffer -> dst.  The first barrier also
// orders this unit's first shared writes after the previous unit's last shared reads.  With
// DST_SMEM the last stage writes the shared buffer too (followed by a barrier), for an epilogue.
// PW: pad elements per 16 in the shared buffer (1; 2 keeps float pairs 16-byte aligned for cp.async).
// ST: tw is the stage-twiddle table (column passes) rather than the length-n table (row passes,
// whose tighter register budget the row loads do not fit)
template <typename T, int DIR, bool DST_SMEM, bool ST, int PW = 1, int SH = 4, class Src, class Dst>
__device__ __forceinline__ void reg_fft(cplx<T>* buf, const FftPlan& fp, int lb, const cplx<T>* tw, const Src& gsrc,
                                        const Dst& gdst) {
  const ShBuf<T, PW, SH> ssrc{buf, lb}, sdst{buf, lb};
  const int S = fp.nstages;
  if (S == 1) {
    // in place in HBM as well (the column pass and the inverse row pass overwrite their input)
    if (DST_SMEM) {
      reg_stage_any<T, DIR, ST>(fp, 0, 1, lb, tw, gsrc, sdst, true);
      __syncthreads();
    } else {
      reg_stage_any<T, DIR, ST>(fp, 0, 1, lb, tw, gsrc, gdst, true);
    }
    return;
  }
  reg_stage_any<T, DIR, ST>(fp, 0, 1, lb, tw, gsrc, sdst, true);
  __syncthreads();
  int Ns = fp.radix[0];
  for (int s = 1; s < S - 1; ++s) {
    reg_stage_any<T, DIR, ST>(fp, s, Ns, lb, tw, ssrc, sdst, true);
    __syncthreads();
    Ns *= fp.radix[s];
  }
  if (DST_SMEM) {
    reg_stage_any<T, DIR, ST>(fp, S - 1, Ns, lb, tw, ssrc, sdst, true);
    __syncthreads();
  } else {
    reg_stage_any<T, DIR, ST>(fp, S - 1, Ns, lb, tw, ssrc, gdst, false);
  }
}

constexpr int kRegMaxThreads = 512;
#define DPS_REG_FFT_BOUNDS __launch_bounds__(kRegMaxThreads, sizeof(T) == 4 ? 2 : 1)

// Every stage but the last of a register-staged transform (at least two stages), into the shared
// buffer; ends with a block barrier, so the last stage may read the buffer.
template <typename T, int DIR, class Src>
__device__ __forceinline__ void reg_fft_head(cplx<T>* buf, const FftPlan& fp, const cplx<T>* tw, const Src& gsrc) {
  const ShBuf<T, 1> sb{buf, 0};
  reg_stage_any<T, DIR, false>(fp, 0, 1, 0, tw, gsrc, sb, true);
  __syncthreads();
  int Ns = fp.radix[0];
  for (int s = 1; s < fp.nstages - 1; ++s) {
    reg_stage_any<T, DIR, false>(fp, s, Ns, 0, tw, sb, sb, true);
    __syncthreads();
    Ns *= fp.radix[s];
  }
}

// The half-spectrum split of two packed real rows: X0_k = (z_k + conj z_{n-k}) / 2 and
// X1_k = (z_k - conj z_{n-k}) / (2i), given z_k and zn = z_{n-k}.
template <typename T>
__device__ __forceinline__ void split_store(cplx<T>* c0, cplx<T>* c1, bool has1, int k, cplx<T> zk, cplx<T> zn) {
  const T half = (T)0.5;
  const cplx<T> zm = conjg(zn);
  c0[k] = scl(zk + zm, half);
  if (has1) {
    const cplx<T> d = zk - zm;
    c1[k] = mk<T>(half * d.y, -half * d.x);
  }
}

// The last stage of the forward row transform (radix R even, span Ns = n / R a multiple of 32)
// fused with the half-spectrum split, so the transform never returns to shared memory.  Butterfly
// jj of the last stage yields z_k for k = jj + Ns r (r < R); the conjugate partner of k is
// n - k = (Ns - jj) + Ns (R - 1 - r), a value of butterfly Ns - jj.  In warp w, lanes 0-15 take
// butterflies x = 16 w + lane and lanes 16-31 their partners Ns - x (Ns / 2 in place of Ns - 0:
// butterflies 0 and Ns / 2 are their own partners), so a lane receives its partner's values by a
// shuffle with lane ^ 16, and every lane writes its values k <= n / 2 of both half spectra.
template <typename T, int R>
__device__ __forceinline__ void r2c_last_split(const cplx<T>* buf, const FftPlan& fp, const cplx<T>* __restrict__ tw,
                                               cplx<T>* c0, cplx<T>* c1, bool has1) {
  static_assert(R % 2 == 0, "the split pairs the outputs of an even radix");
  const int Ns = fp.n / R, t = threadIdx.x;
  if (t >= Ns) return;  // whole warps
  const int jj = pair_butterfly(t, Ns);
  cplx<T> v[R];
  const int p0 = pad16(jj), sp = Ns + (Ns >> 4);  // Ns is a multiple of 16: the padding is linear in r
#pragma unroll
  for (int r = 0; r < R; ++r) v[r] = buf[p0 + r * sp];
#pragma unroll
  for (int r = 1; r < R; ++r) v[r] = v[r] * tw[jj * r];  // W_{Ns R}^{jj r} = W_n^{jj r}
  Dft<T, R, -1>::run(v);
  const bool self0 = jj == 0, selfh = 2 * jj == Ns;
#pragma unroll
  for (int r = 0; r < R / 2; ++r) {
    cplx<T> q = v[R - 1 - r];
    q.x = __shfl_xor_sync(0xffffffffu, q.x, 16);
    q.y = __shfl_xor_sync(0xffffffffu, q.y, 16);
    const cplx<T> zn = self0 ? v[(R - r) % R] : (selfh ? v[R - 1 - r] : q);
    split_store(c0, c1, has1, jj + Ns * r, v[r], zn);
  }
  if (self0) split_store(c0, c1, has1, fp.n / 2, v[R / 2], v[R / 2]);
}

template <typename T>
__device__ __forceinline__ void r2c_last_split_any(const cplx<T>* buf, const FftPlan& fp, const cplx<T>* tw,
                                                   cplx<T>* c0, cplx<T>* c1, bool has1) {
  switch (fp.radix[fp.nstages - 1]) {
    case 16: r2c_last_split<T, 16>(buf, fp, tw, c0, c1, has1); break;
    case 12: r2c_last_split<T, 12>(buf, fp, tw, c0, c1, has1); break;
    case 8: r2c_last_split<T, 8>(buf, fp, tw, c0, c1, has1); break;
    case 4: r2c_last_split<T, 4>(buf, fp, tw, c0, c1, has1); break;
    default: r2c_last_split<T, 2>(buf, fp, tw, c0, c1, has1); break;
  }
}

// whether a row factorisation takes the fused last stage (r2c_last_split)
bool r2c_split_ok(const FftPlan& fp) {
  if (fp.nstages < 2) return false;
  const int R = fp.radix[fp.nstages - 1];
  return R % 2 == 0 && R <= 16 && (fp.n / R) % 32 == 0;
}

// Row pass, forward, register-staged: two real rows packed as z = r0 + i r1, then the half-spectrum
// split (SPLIT: in the last stage's registers, r2c_last_split; else from the shared buffer).
template <typename T, bool SPLIT>
__global__ void DPS_REG_FFT_BOUNDS row_r2c_reg_kernel(Geometry g, FftPlan fp, const cplx<T>* __restrict__ tw,
                                                      T* __restrict__ grid, const int* __restrict__ zrange) {
  extern __shared__ __align__(16) unsigned char smraw[];
  cplx<T>* buf = reinterpret_cast<cplx<T>*>(smraw);
  const int nx = g.nx;
  const UnitMap um(g, zrange, (g.ny + 1) / 2);
  const size_t rowlen = (size_t)2 * g.pitch;
  const T half = (T)0.5;
  for (long long u = blockIdx.x; u < um.total; u += gridDim.x) {
    int f, c, j;
    um.at(u, f, c, j);
    const bool has1 = 2 * j + 1 < g.ny;
    T* row0 = grid + ((size_t)(f * g.nz + c) * g.ny + 2 * j) * rowlen;
    const T* row1 = row0 + rowlen;
    auto src = [&](int e, int) { return mk<T>(row0[e], has1 ? row1[e] : (T)0); };
    cplx<T>* c0 = reinterpret_cast<cplx<T>*>(row0);
    cplx<T>* c1 = reinterpret_cast<cplx<T>*>(row0 + rowlen);
    if (SPLIT) {
      // the next unit's first stage writes the buffer only after a block barrier (reg_stage), by
      // which time every thread has read its last-stage inputs
      reg_fft_head<T, -1>(buf, fp, tw, src);
      r2c_last_split_any<T>(buf, fp, tw, c0, c1, has1);
      continue;
    }
    reg_fft<T, -1, true, false>(buf, fp, 0, tw, src, [](int, int, cplx<T>) {});
    for (int k = threadIdx.x; k <= nx / 2; k += blockDim.x) {
      const cplx<T> zk = buf[pad16(k)];
      const cplx<T> zm = conjg(buf[pad16(k == 0 ? 0 : nx - k)]);
      c0[k] = scl(zk + zm, half);
      if (has1) {
        const cplx<T> d = zk - zm;  // (zk - conj z_{-k}) / (2i)
        c1[k] = mk<T>(half * d.y, -half * d.x);
      }
    }
  }
}

// The first stage of the inverse row transform (radix R even, n / R a multiple of 32) reading each
// half-spectrum value once.  Butterfly jj reads z_e, e = jj + (n / R) r, with z_e = X0_e + i X1_e
// for e <= n / 2 and conj X0_{n-e} + i conj X1_{n-e} beyond; n - e is input R - 1 - r of
// butterfly n / R - jj.  With the lane pairing of r2c_last_split (partners in lanes l and l ^ 16,
// butterflies 0 and n / (2 R) their own partners), a lane reads its inputs below n / 2 (r < R / 2),
// forms z_e and z_{n-e}, and hands z_{n-e} to its partner by a shuffle.  The stage then writes the
// shared buffer after a block barrier, as reg_stage does.
template <typename T, int R>
__device__ __forceinline__ void c2r_first_pair(cplx<T>* buf, const FftPlan& fp, const cplx<T>* c0,
                                               const cplx<T>* c1, bool has1) {
  static_assert(R % 2 == 0, "the pairing needs an even radix");
  const int nr = fp.n / R, t = threadIdx.x;
  const bool act = t < nr;  // whole warps
  cplx<T> v[R];  // initialised: an array left undefined on the idle threads' path is not kept in registers
#pragma unroll
  for (int r = 0; r < R; ++r) v[r] = mk<T>((T)0, (T)0);
  int jj = 0;
  if (act) {
    jj = pair_butterfly(t, nr);
#pragma unroll
    for (int r = 0; r < R / 2; ++r) {
      const int k = jj + nr * r;  // below n / 2
      const cplx<T> x0 = c0[k];
      const cplx<T> x1 = has1 ? c1[k] : mk<T>((T)0, (T)0);
      v[r] = x0 + mul_i(x1);
      v[R - 1 - r] = conjg(x0) + mul_i(conjg(x1));  // z_{n-k}, the partner's input R - 1 - r
    }
#pragma unroll
    for (int r = R / 2; r < R; ++r) {  // exchange the upper halves with the partner lane
      v[r].x = __shfl_xor_sync(0xffffffffu, v[r].x, 16);
      v[r].y = __shfl_xor_sync(0xffffffffu, v[r].y, 16);
    }
    if (pair_self(jj, nr)) {  // their own partners (two lanes of the first warp): direct reads
#pragma unroll
      for (int r = R / 2; r < R; ++r) {
        const int e = jj + nr * r;  // at least n / 2
        const int k = e == fp.n / 2 ? e : fp.n - e;
        const cplx<T> x0 = c0[k];
        const cplx<T> x1 = has1 ? c1[k] : mk<T>((T)0, (T)0);
        v[r] = e == fp.n / 2 ? x0 + mul_i(x1) : conjg(x0) + mul_i(conjg(x1));
      }
    }
    Dft<T, R, +1>::run(v);
  }
  __syncthreads();
  if (act) {
#pragma unroll
    for (int r = 0; r < R; ++r) buf[pad16(jj * R + r)] = v[r];
  }
}

template <typename T>
__device__ __forceinline__ void c2r_first_pair_any(cplx<T>* buf, const FftPlan& fp, const cplx<T>* c0,
                                                   const cplx<T>* c1, bool has1) {
  switch (fp.radix[0]) {
    case 16: c2r_first_pair<T, 16>(buf, fp, c0, c1, has1); break;
    case 12: c2r_first_pair<T, 12>(buf, fp, c0, c1, has1); break;
    case 8: c2r_first_pair<T, 8>(buf, fp, c0, c1, has1); break;
    case 4: c2r_first_pair<T, 4>(buf, fp, c0, c1, has1); break;
    default: c2r_first_pair<T, 2>(buf, fp, c0, c1, has1); break;
  }
}

// whether a row factorisation takes the paired first stage (c2r_first_pair)
bool c2r_pair_ok(const FftPlan& fp) {
  if (fp.nstages < 2) return false;
  const int R = fp.radix[0];
  return R % 2 == 0 && R <= 16 && (fp.n / R) % 32 == 0;
}

// Stages 1 .. S - 1 of a register-staged transform from the shared buffer (after the first stage
// and a block barrier), the last writing through dst.
template <typename T, int DIR, class Dst>
__device__ __forceinline__ void reg_fft_tail(cplx<T>* buf, const FftPlan& fp, const cplx<T>* tw, const Dst& gdst) {
  const ShBuf<T, 1> sb{buf, 0};
  int Ns = fp.radix[0];
  for (int s = 1; s < fp.nstages - 1; ++s) {
    reg_stage_any<T, DIR, false>(fp, s, Ns, 0, tw, sb, sb, true);
    __syncthreads();
    Ns *= fp.radix[s];
  }
  reg_stage_any<T, DIR, false>(fp, fp.nstages - 1, Ns, 0, tw, sb, gdst, false);
}

// Row pass, inverse, register-staged: z_k = X0_k + i X1_k over the Hermitian extension, one FFT
// (PAIR: the first stage reads each half-spectrum value once, c2r_first_pair).
template <typename T, bool PAIR>
__global__ void DPS_REG_FFT_BOUNDS row_c2r_reg_kernel(Geometry g, FftPlan fp, const cplx<T>* __restrict__ tw,
                                                      T* __restrict__ grid, const int* __restrict__ zrange) {
  extern __shared__ __align__(16) unsigned char smraw[];
  cplx<T>* buf = reinterpret_cast<cplx<T>*>(smraw);
  const int nx = g.nx;
  const UnitMap um(g, zrange, (g.ny + 1) / 2);
  const size_t rowlen = (size_t)2 * g.pitch;
  for (long long u = blockIdx.x; u < um.total; u += gridDim.x) {
    int f, c, j;
    um.at(u, f, c, j);
    const bool has1 = 2 * j + 1 < g.ny;
    T* row0 = grid + ((size_t)(f * g.nz + c) * g.ny + 2 * j) * rowlen;
    T* row1 = row0 + rowlen;
    const cplx<T>* c0 = reinterpret_cast<const cplx<T>*>(row0);
    const cplx<T>* c1 = reinterpret_cast<const cplx<T>*>(row1);
    if (PAIR) {
      c2r_first_pair_any<T>(buf, fp, c0, c1, has1);
      __syncthreads();
      reg_fft_tail<T, +1>(buf, fp, tw, [&](int a, int, cplx<T> v) {
        row0[a] = v.x;
        if (has1) row1[a] = v.y;
      });
      continue;
    }
    reg_fft<T, +1, false, false>(
        buf, fp, 0, tw,
        [&](int e, int) {
          const bool lo = e <= nx / 2;
          const int k = lo ? e : nx - e;
          const cplx<T> x0 = c0[k];
          const cplx<T> x1 = has1 ? c1[k] : mk<T>((T)0, (T)0);
          return lo ? x0 + mul_i(x1) : conjg(x0) + mul_i(conjg(x1));
        },
        [&](int a, int, cplx<T> v) {
          row0[a] = v.x;
          if (has1) row1[a] = v.y;
        });
  }
}

// Column pass, register-staged: cw = 2^lcw adjacent x-wavenumber columns of one plane, along y.
template <typename T, int DIR>
__global__ void DPS_REG_FFT_BOUNDS col_reg_kernel(Geometry g, FftPlan fp, const cplx<T>* __restrict__ tw,
                                                  cplx<T>* __restrict__ grid, const int* __restrict__ zrange, int lcw,
                                                  int kxs, int kxe) {
  extern __shared__ __align__(16) unsigned char smraw[];
  cplx<T>* buf = reinterpret_cast<cplx<T>*>(smraw);
  const int cw = 1 << lcw;
  const UnitMap um(g, zrange, (kxe - kxs + cw - 1) >> lcw);
  for (long long u = blockIdx.x; u < um.total; u += gridDim.x) {
    int f, c, j;
    um.at(u, f, c, j);
    const int kx0 = kxs + (j << lcw);
    const int ncols = min(cw, kxe - kx0);
    cplx<T>* base = grid + (size_t)(f * g.nz + c) * g.ny * g.pitch + kx0;
    reg_fft<T, DIR, false, true>(
        buf, fp, lcw, tw,
        [&](int y, int b) { return b < ncols ? base[(size_t)y * g.pitch + b] : mk<T>((T)0, (T)0); },
        [&](int y, int b, cplx<T> v) {
          if (b < ncols) base[(size_t)y * g.pitch + b] = v;
        });
  }
}

// Column pass, prefetched and register-staged: two unit buffers in shared memory; while the block
// transforms one in place (one butterfly per thread and stage, the last stage writing HBM), cp.async
// fills the other with the next unit.  The two buffers take most of the SM's shared memory, so a
// unit can be 4 columns x 3072 rows (a full 32-byte sector per row, half the requests of 2 columns).
// padding of the unit buffers: float, 2 values per 32 (pairs stay 16-byte aligned for cp.async, and
// the first stage's stores, 64 values apart across a warp, spread over the banks 2-way instead of
// 4-way with 2 per 16); double, 1 per 16
template <typename T>
__host__ __device__ constexpr int pipe_pad() { return sizeof(cplx<T>) == 8 ? 2 : 1; }
template <typename T>
__host__ __device__ constexpr int pipe_pad_shift() { return sizeof(cplx<T>) == 8 ? 5 : 4; }
constexpr int kPipeMaxThreadsF = 1024, kPipeMaxThreadsD = 512;

template <typename T, int DIR>
__global__ void __launch_bounds__(sizeof(T) == 4 ? kPipeMaxThreadsF : kPipeMaxThreadsD, 1)
    col_pipe_kernel(Geometry g, FftPlan fp, const cplx<T>* __restrict__ tw, cplx<T>* __restrict__ grid,
                    const int* __restrict__ zrange, int lcw, int kxs, int kxe) {
  extern __shared__ __align__(16) unsigned char smraw[];
  constexpr int PW = pipe_pad<T>(), SH = pipe_pad_shift<T>();
  const int cw = 1 << lcw;
  const int pts = g.ny << lcw;
  const int blen = pts + PW * (pts >> SH) + PW;
  cplx<T>* const buf0 = reinterpret_cast<cplx<T>*>(smraw);
  cplx<T>* const buf1 = buf0 + blen;
  const UnitMap um(g, zrange, (kxe - kxs + cw - 1) >> lcw);
  auto base_of = [&](long long u, int& ncols) {
    int f, c, j;
    um.at(u, f, c, j);
    const int kx0 = kxs + (j << lcw);
    ncols = min(cw, kxe - kx0);
    return grid + (size_t)(f * g.nz + c) * g.ny * g.pitch + kx0;
  };
  auto issue = [&](long long u, cplx<T>* dst) {
    int ncols;
    const cplx<T>* base = base_of(u, ncols);
    const bool wide = ncols == cw && (cw * sizeof(cplx<T>)) % 16 == 0 && (reinterpret_cast<size_t>(base) & 15) == 0;
    if (wide) {
      constexpr int E = sizeof(cplx<T>) == 8 ? 2 : 1;  // elements per 16 bytes
      const int per = cw / E;
      for (int t = threadIdx.x; t < g.ny * per; t += blockDim.x) {
        const int y = t / per, q = t - y * per;
        cp_async16(dst + padw<PW, SH>((y << lcw) + q * E), base + (size_t)y * g.pitch + q * E);
      }
    } else {
      for (int t = threadIdx.x; t < pts; t += blockDim.x) {
        const int y = t >> lcw, b = t & (cw - 1);
        if (b < ncols) async_elem(dst + padw<PW, SH>(t), base + (size_t)y * g.pitch + b);
        else dst[padw<PW, SH>(t)] = mk<T>((T)0, (T)0);  // columns past the x range transform as zeros
      }
    }
    cp_commit();
  };
  long long u = blockIdx.x;
  bool odd = false;
  if (u < um.total) issue(u, buf0);
  for (; u < um.total; u += gridDim.x, odd = !odd) {
    cplx<T>* const cur = odd ? buf1 : buf0;
    cplx<T>* const nxt = odd ? buf0 : buf1;
    int ncols;
    cplx<T>* base = base_of(u, ncols);
    cp_wait_all();
    __syncthreads();  // this unit staged; every thread is done with the previous unit (in nxt)
    if (u + gridDim.x < um.total) issue(u + gridDim.x, nxt);
    reg_fft<T, DIR, false, true, PW, SH>(
        cur, fp, lcw, tw,
        ShBuf<T, PW, SH>{cur, lcw},
        [&](int y, int b, cplx<T> v) {
          if (b < ncols) base[(size_t)y * g.pitch + b] = v;
        });
  }
  cp_wait_all();  // no copy outstanding at exit
}

// ---- TMA-staged column pass ----
// As col_pipe_kernel, but the next unit arrives by TMA: one thread arms the buffer's mbarrier with
// the unit's byte count and issues ny / bh box loads (2 cw reals x bh rows each) of the grid's
// tensor map into the buffer, densely ([y][b]); the first FFT stage reads that dense layout and its
// in-place writes (after the stage's barrier) use the padded one.  Every wait is bounded (about a
// second): on expiry the block records kStatTimeout, waits (bounded again) for its copies in flight
// and leaves.  `withhold` (failure injection for tests) arms each buffer's barrier but issues no box
// load, so the first wait runs out with no copy in flight.

__device__ __forceinline__ void mbar_init(uint64_t* bar, unsigned count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;\n" ::"r"(smem_u32(bar)), "r"(count) : "memory");
}
__device__ __forceinline__ void mbar_expect_tx(uint64_t* bar, unsigned bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;\n" ::"r"(smem_u32(bar)), "r"(bytes) : "memory");
}
// bounded wait for the phase with the given parity to complete; false after about 2^31 cycles
__device__ __forceinline__ bool mbar_wait(uint64_t* bar, unsigned parity) {
  const long long t0 = clock64();
  for (;;) {
    unsigned done;
    asm volatile(
        "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}\n"
        : "=r"(done)
        : "r"(smem_u32(bar)), "r"(parity)
        : "memory");
    if (done) return true;
    if (clock64() - t0 > (1LL << 31)) return false;
  }
}
__device__ __forceinline__ void tma_load_2d(void* dst, const CUtensorMap* map, int x, int y, uint64_t* bar) {
  asm volatile(
      "cp.async.bulk.tensor.2d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3}], [%4];\n" ::"r"(
          smem_u32(dst)),
      "l"(reinterpret_cast<uint64_t>(map)), "r"(x), "r"(y), "r"(smem_u32(bar))
      : "memory");
}

// unit buffer length in values: the padded layout, rounded up to 128 bytes (TMA destinations)
template <typename T>
__host__ __device__ __forceinline__ int tma_buf_len(int points) {
  const int n = points + pipe_pad<T>() * (points >> pipe_pad_shift<T>()) + pipe_pad<T>();
  const int q = 128 / (int)sizeof(cplx<T>);
  return (n + q - 1) / q * q;
}

template <typename T, int DIR>
__global__ void __launch_bounds__(sizeof(T) == 4 ? kPipeMaxThreadsF : kPipeMaxThreadsD, 1)
    col_tma_kernel(const __grid_constant__ CUtensorMap tmap, Geometry g, FftPlan fp, const cplx<T>* __restrict__ tw,
                   cplx<T>* __restrict__ grid, const int* __restrict__ zrange, int* __restrict__ status, int lcw,
                   int kxs, int kxe, int bh, int withhold) {
  extern __shared__ __align__(16) unsigned char smraw[];  // realigned to 128 bytes below
  constexpr int PW = pipe_pad<T>(), SH = pipe_pad_shift<T>();
  const int cw = 1 << lcw;
  const int pts = g.ny << lcw;
  const int blen = tma_buf_len<T>(pts);
  cplx<T>* const buf0 = reinterpret_cast<cplx<T>*>((reinterpret_cast<uintptr_t>(smraw) + 127) & ~(uintptr_t)127);
  cplx<T>* const buf1 = buf0 + blen;
  uint64_t* const bars = reinterpret_cast<uint64_t*>(buf1 + blen);
  const UnitMap um(g, zrange, (kxe - kxs + cw - 1) >> lcw);
  const unsigned bytes = (unsigned)pts * (unsigned)sizeof(cplx<T>);
  if (threadIdx.x == 0) {
    mbar_init(&bars[0], 1);
    mbar_init(&bars[1], 1);
    asm volatile("fence.mbarrier_init.release.cluster;\n" ::: "memory");
  }
  __syncthreads();
  auto issue = [&](long long u, int w) {  // thread 0
    int f, c, j;
    um.at(u, f, c, j);
    const int kx0 = kxs + (j << lcw);
    const int y0 = (f * g.nz + c) * g.ny;
    cplx<T>* dst = w ? buf1 : buf0;
    // the buffer's last contents were written by the generic proxy (the previous unit's stages)
    asm volatile("fence.proxy.async.shared::cta;\n" ::: "memory");
    mbar_expect_tx(&bars[w], bytes);
    if (withhold) return;
    for (int r0 = 0; r0 < g.ny; r0 += bh) tma_load_2d(dst + (r0 << lcw), &tmap, 2 * kx0, y0 + r0, &bars[w]);
  };
  unsigned phase = 0;  // bit w: parity of the next completion of barrier w
  long long u = blockIdx.x;
  if (u < um.total && threadIdx.x == 0) issue(u, 0);
  for (int w = 0; u < um.total; u += gridDim.x, w ^= 1) {
    cplx<T>* const cur = w ? buf1 : buf0;
    const bool ok = mbar_wait(&bars[w], (phase >> w) & 1u);
    phase ^= 1u << w;
    // also: every thread is done with the previous unit (the other buffer)
    if (__syncthreads_or(!ok)) {
      if (threadIdx.x == 0) {
        atomicOr(status, kStatTimeout);
        mbar_wait(&bars[w], ((phase >> w) & 1u) ^ 1u);  // give this unit's copies a second chance to land
      }
      return;
    }
    if (u + gridDim.x < um.total && threadIdx.x == 0) issue(u + gridDim.x, w ^ 1);
    int f, c, j;
    um.at(u, f, c, j);
    const int kx0 = kxs + (j << lcw);
    const int ncols = min(cw, kxe - kx0);
    cplx<T>* base = grid + (size_t)(f * g.nz + c) * g.ny * g.pitch + kx0;
    reg_fft<T, DIR, false, true, PW, SH>(cur, fp, lcw, tw, ShBuf<T, 0, SH>{cur, lcw},
                                         [&](int y, int b, cplx<T> v) {
                                           if (b < ncols) base[(size_t)y * g.pitch + b] = v;
                                         });
  }
}

size_t padded_bytes(int n, size_t esz) { return (size_t)(n + (n >> 4) + 1) * esz; }

template <typename T>
size_t row_r2c_smem(const Geometry& g) {
  return (size_t)2 * staged_len(g.nx) * sizeof(T) + 2 * padded_bytes(g.nx, sizeof(cplx<T>)) +
         (size_t)g.nx * sizeof(cplx<T>);
}
template <typename T>
size_t row_c2r_smem(const Geometry& g) {
  return (size_t)2 * ((g.nx / 2 + 2) & ~1) * sizeof(cplx<T>) + 2 * padded_bytes(g.nx, sizeof(cplx<T>)) +
         (size_t)g.nx * sizeof(cplx<T>);
}
template <typename T>
size_t col_smem(const Geometry& g, int l) {
  return (size_t)(g.ny << l) * sizeof(cplx<T>) + 2 * padded_bytes(g.ny << l, sizeof(cplx<T>)) +
         (size_t)g.ny * sizeof(cplx<T>);
}

constexpr int kFftMaxThreads = 512;

// threads for a transform of `points` values: at most kFftPer per thread, whole warps
int fft_threads(int points) { return std::max(32, (points + kFftPer * 32 - 1) / (kFftPer * 32) * 32); }

// log2 of the column block: the widest (at most 8 columns) within the thread limit whose staging,
// work and twiddle buffers fit in 190 KB of shared memory
template <typename T>
int col_lwidth(const Plan& p) {
  for (int l = 3; l > 0; --l)
    if (fft_threads(p.g.ny << l) <= kFftMaxThreads && col_smem<T>(p.g, l) <= 190 * 1024) return l;
  return 0;
}

template <typename KernelT>
int resident_grid(KernelT kernel, int threads, size_t smem, int device) {
  int per_sm = 0, sms = 0;
  cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kernel, threads, smem);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, device);
  return std::max(1, per_sm) * std::max(1, sms);
}

// threads of the register-staged variant for `points` = n 2^lb values: one per butterfly of the
// stage with the most butterflies, whole warps
int reg_threads(const FftPlan& fp, int lb) {
  int m = 0;
  for (int s = 0; s < fp.nstages; ++s) m = std::max(m, (fp.n << lb) / fp.radix[s]);
  return (m + 31) / 32 * 32;
}

template <typename T>
size_t reg_smem(int points) { return padded_bytes(points, sizeof(cplx<T>)); }

// the register-staged variant fits: thread limit, and the two resident blocks per SM (float) its
// register budget was compiled for share the SM's shared memory
template <typename T>
bool reg_fits(const FftPlan& fp, int lb) {
  return reg_threads(fp, lb) <= kRegMaxThreads && reg_smem<T>(fp.n << lb) <= 100 * 1024;
}

}  // namespace

template <typename T>
size_t pipe_smem(int points) {
  constexpr int PW = pipe_pad<T>(), SH = pipe_pad_shift<T>();
  return (size_t)2 * (points + PW * (points >> SH) + PW) * sizeof(cplx<T>);
}

template <typename T>
bool pipe_fits(const FftPlan& fp, int lb) {
  const int maxth = sizeof(T) == 4 ? kPipeMaxThreadsF : kPipeMaxThreadsD;
  return reg_threads(fp, lb) <= maxth && pipe_smem<T>(fp.n << lb) <= 224 * 1024;
}

template <typename T>
size_t tma_smem(int points) { return 128 + (size_t)2 * tma_buf_len<T>(points) * sizeof(cplx<T>) + 16; }

// rows per TMA box: the largest divisor of ny up to 256 whose boxes keep 128-byte alignment in the
// unit buffer; 0 if there is none
template <typename T>
int tma_box_rows(int ny, int lcw) {
  for (int h = std::min(ny, 256); h >= 1; --h)
    if (ny % h == 0 && ((size_t)h * (1u << lcw) * sizeof(cplx<T>)) % 128 == 0) return h;
  return 0;
}

// the grid as a rank-2 tensor of reals (2 pitch per row, nfields nz ny rows) with boxes of
// 2^lcw complex columns x bh rows; false when cuTensorMapEncodeTiled cannot be obtained or refuses it
template <typename T>
bool encode_col_tmap(Plan& p, int lcw, int bh) {
  void* fn = nullptr;
  cudaDriverEntryPointQueryResult q;
  if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &fn, 12000, cudaEnableDefault, &q) != cudaSuccess ||
      q != cudaDriverEntryPointSuccess || fn == nullptr)
    return false;
  auto encode = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(fn);
  const Geometry& g = p.g;
  const cuuint64_t dims[2] = {(cuuint64_t)2 * g.pitch, (cuuint64_t)g.nfields * g.nz * g.ny};
  const cuuint64_t strides[1] = {(cuuint64_t)2 * g.pitch * sizeof(T)};
  const cuuint32_t box[2] = {(cuuint32_t)(2u << lcw), (cuuint32_t)bh};
  const cuuint32_t estr[2] = {1, 1};
  CUtensorMap* map = reinterpret_cast<CUtensorMap*>(p.col_tmap);
  return encode(map, sizeof(T) == 4 ? CU_TENSOR_MAP_DATA_TYPE_FLOAT32 : CU_TENSOR_MAP_DATA_TYPE_FLOAT64, 2, p.grid,
                dims, strides, box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE,
                CU_TENSOR_MAP_L2_PROMOTION_NONE, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

template <typename T>
int fft_set_col_width(Plan& p, int lcw, int reg) {
  if (lcw < 0 || lcw > 3 || reg < 0 || reg > 3) return 0;
  if (reg == 3) {
    const int maxth = sizeof(T) == 4 ? kPipeMaxThreadsF : kPipeMaxThreadsD;
    const int th = reg_threads(p.fyr, lcw);
    const size_t sm = tma_smem<T>(p.g.ny << lcw);
    const int bh = tma_box_rows<T>(p.g.ny, lcw);
    // box rows of 16-byte multiples; a block never reads past the padded row (pitch is a multiple
    // of 32 columns and a block starts at a multiple of its width)
    if (th > maxth || sm > 224 * 1024 || bh == 0 || ((2u << lcw) * sizeof(T)) % 16 != 0) return 0;
    if (!encode_col_tmap<T>(p, lcw, bh)) return 0;
    p.col_lcw = lcw;
    p.fft_reg[1] = 3;
    p.col_tma_rows = bh;
    p.fft_grid[2] = resident_grid(col_tma_kernel<T, -1>, th, sm, p.device);
    p.fft_grid[3] = resident_grid(col_tma_kernel<T, +1>, th, sm, p.device);
    return 1;
  }
  if (reg == 2) {
    if (!pipe_fits<T>(p.fyr, lcw)) return 0;
    const int th = reg_threads(p.fyr, lcw);
    const size_t sm = pipe_smem<T>(p.g.ny << lcw);
    p.col_lcw = lcw;
    p.fft_reg[1] = 2;
    p.fft_grid[2] = resident_grid(col_pipe_kernel<T, -1>, th, sm, p.device);
    p.fft_grid[3] = resident_grid(col_pipe_kernel<T, +1>, th, sm, p.device);
    return 1;
  }
  if (reg) {
    if (!reg_fits<T>(p.fyr, lcw)) return 0;
    const int th = reg_threads(p.fyr, lcw);
    const size_t sm = reg_smem<T>(p.g.ny << lcw);
    p.col_lcw = lcw;
    p.fft_reg[1] = 1;
    p.fft_grid[2] = resident_grid(col_reg_kernel<T, -1>, th, sm, p.device);
    p.fft_grid[3] = resident_grid(col_reg_kernel<T, +1>, th, sm, p.device);
    return 1;
  }
  const size_t col = col_smem<T>(p.g, lcw);
  const int tcol = fft_threads(p.g.ny << lcw);
  if (tcol > kFftMaxThreads || col > 220 * 1024) return 0;
  p.col_lcw = lcw;
  p.fft_reg[1] = 0;
  p.fft_grid[2] = resident_grid(col_kernel<T, -1>, tcol, col, p.device);
  p.fft_grid[3] = resident_grid(col_kernel<T, +1>, tcol, col, p.device);
  return 1;
}

template <typename T>
int fft_set_row_variant(Plan& p, int reg) {
  if (reg) {
    if (!reg_fits<T>(p.fxr, 0)) return 0;
    const int th = reg_threads(p.fxr, 0);
    const size_t sm = reg_smem<T>(p.g.nx);
    p.fft_reg[0] = 1;
    p.fft_grid[0] = r2c_split_ok(p.fxr) ? resident_grid(row_r2c_reg_kernel<T, true>, th, sm, p.device)
                                         : resident_grid(row_r2c_reg_kernel<T, false>, th, sm, p.device);
    p.fft_grid[1] = c2r_pair_ok(p.fxr) ? resident_grid(row_c2r_reg_kernel<T, true>, th, sm, p.device)
                                        : resident_grid(row_c2r_reg_kernel<T, false>, th, sm, p.device);
    return 1;
  }
  const size_t r2c = row_r2c_smem<T>(p.g), c2r = row_c2r_smem<T>(p.g);
  const int trow = fft_threads(p.g.nx);
  if (trow > kFftMaxThreads || r2c > 220 * 1024 || c2r > 220 * 1024) return 0;
  p.fft_reg[0] = 0;
  p.fft_grid[0] = resident_grid(row_r2c_kernel<T>, trow, r2c, p.device);
  p.fft_grid[1] = resident_grid(row_c2r_kernel<T>, trow, c2r, p.device);
  return 1;
}

// Default shapes, from measurements on rollers and slit grids (3072^2, 768^2, 384^2): the
// register-staged row pass only for long float rows whose stages keep at least 3/4 of the block
// busy (3072 = 16 x 16 x 12: 10 % faster than the shared-memory-staged pass; 768 = 16 x 16 x 3 and
// 384 = 16 x 12 x 2 leave most threads idle in the radix-16 stages and run 1.5-2.5x slower, as does
// FP64).  Columns: the width of a block's per-row piece decides (3072 rows, mixed: 2 columns
// shared-memory-staged 18.1 ms per pass pair, 4 columns prefetched register-staged 14.5 ms, the
// latter at 2 columns 23.6 ms), so the prefetched register-staged pass where its two buffers fit a
// wider block than the staged pass's three, else the staged pass at its widest; the register-staged
// pass without prefetch (loads exposed; 1.3-1.5x slower at equal width) only by hand or autotuning.
template <typename T>
bool reg_rows_default(const FftPlan& fp) {
  if (sizeof(T) != 4 || fp.n < 2048 || !reg_fits<T>(fp, 0)) return false;
  int rmin = fp.radix[0], rmax = fp.radix[0];
  for (int s = 1; s < fp.nstages; ++s) {
    rmin = std::min(rmin, fp.radix[s]);
    rmax = std::max(rmax, fp.radix[s]);
  }
  return 3 * rmax <= 4 * rmin;
}

template <typename T>
int fft_smem_ok(Plan& p) {
  if (!allow_smem(row_r2c_kernel<T>) || !allow_smem(row_c2r_kernel<T>) || !allow_smem(col_kernel<T, -1>) ||
      !allow_smem(col_kernel<T, +1>) || !allow_smem(row_r2c_reg_kernel<T, false>) ||
      !allow_smem(row_r2c_reg_kernel<T, true>) || !allow_smem(row_c2r_reg_kernel<T, false>) ||
      !allow_smem(row_c2r_reg_kernel<T, true>) ||
      !allow_smem(col_reg_kernel<T, -1>) || !allow_smem(col_reg_kernel<T, +1>) ||
      !allow_smem(col_pipe_kernel<T, -1>) || !allow_smem(col_pipe_kernel<T, +1>) ||
      !allow_smem(col_tma_kernel<T, -1>) || !allow_smem(col_tma_kernel<T, +1>))
    return 0;
  const bool rr = reg_rows_default<T>(p.fxr);
  if (!fft_set_row_variant<T>(p, rr ? 1 : 0) && !fft_set_row_variant<T>(p, rr ? 0 : 1)) return 0;
  // columns: the prefetched register-staged pass when it fits a wider block than the staged one,
  // prefetched by TMA where a box shape fits (3072^2: 12.2 -> 10.7 ms per pass pair), else cp.async
  const int ls = col_lwidth<T>(p);
  for (int l = 3; l > ls; --l)
    if (fft_set_col_width<T>(p, l, 3) || fft_set_col_width<T>(p, l, 2)) return 1;
  // at the staged pass's width, TMA on long columns (768 rows, 8 columns: 0.78 -> 0.70 ms per pass
  // pair; 384 rows: 0.57 staged against 0.66, the units too short for the per-unit barrier work)
  if (p.g.ny >= 512 && fft_set_col_width<T>(p, ls, 3)) return 1;
  if (fft_set_col_width<T>(p, ls, 0)) return 1;
  for (int l = 3; l >= 0; --l)
    if (fft_set_col_width<T>(p, l, 1)) return 1;
  return 0;
}

template <typename T>
void launch_fft_rows(const Plan& p, int dir, cudaStream_t s) {
  const Geometry& g = p.g;
  const cplx<T>* twx = reinterpret_cast<const cplx<T>*>(p.tab.twx);
  if (p.fft_reg[0]) {
    const int th = reg_threads(p.fxr, 0);
    const size_t sm = reg_smem<T>(g.nx);
    T* grid = reinterpret_cast<T*>(p.grid);
    if (dir < 0 && r2c_split_ok(p.fxr))
      row_r2c_reg_kernel<T, true><<<p.fft_grid[0], th, sm, s>>>(g, p.fxr, twx, grid, p.zrange);
    else if (dir < 0)
      row_r2c_reg_kernel<T, false><<<p.fft_grid[0], th, sm, s>>>(g, p.fxr, twx, grid, p.zrange);
    else if (c2r_pair_ok(p.fxr))
      row_c2r_reg_kernel<T, true><<<p.fft_grid[1], th, sm, s>>>(g, p.fxr, twx, grid, p.zrange);
    else
      row_c2r_reg_kernel<T, false><<<p.fft_grid[1], th, sm, s>>>(g, p.fxr, twx, grid, p.zrange);
    return;
  }
  const int th = fft_threads(g.nx);
  if (dir < 0)
    row_r2c_kernel<T><<<p.fft_grid[0], th, row_r2c_smem<T>(g), s>>>(g, p.fx, twx, reinterpret_cast<T*>(p.grid),
                                                                      p.zrange);
  else
    row_c2r_kernel<T><<<p.fft_grid[1], th, row_c2r_smem<T>(g), s>>>(g, p.fx, twx, reinterpret_cast<T*>(p.grid),
                                                                      p.zrange);
}

template <typename T>
void launch_fft_cols(const Plan& p, int dir, int kxs, int kxe, cudaStream_t s) {
  const Geometry& g = p.g;
  const cplx<T>* twy = reinterpret_cast<const cplx<T>*>(p.tab.twy);
  const int lcw = p.col_lcw;
  cplx<T>* grid = reinterpret_cast<cplx<T>*>(p.grid);
  const cplx<T>* tsy = reinterpret_cast<const cplx<T>*>(p.tab.tsy);
  if (p.fft_reg[1] == 3) {
    const int th = reg_threads(p.fyr, lcw);
    const size_t sm = tma_smem<T>(g.ny << lcw);
    const CUtensorMap& map = *reinterpret_cast<const CUtensorMap*>(p.col_tmap);
    if (dir < 0)
      col_tma_kernel<T, -1><<<p.fft_grid[2], th, sm, s>>>(map, g, p.fyr, tsy, grid, p.zrange, p.status, lcw, kxs, kxe,
                                                          p.col_tma_rows, p.inject == 3 ? 1 : 0);
    else
      col_tma_kernel<T, +1><<<p.fft_grid[3], th, sm, s>>>(map, g, p.fyr, tsy, grid, p.zrange, p.status, lcw, kxs, kxe,
                                                          p.col_tma_rows, 0);
    return;
  }
  if (p.fft_reg[1] == 2) {
    const int th = reg_threads(p.fyr, lcw);
    const size_t sm = pipe_smem<T>(g.ny << lcw);
    if (dir < 0)
      col_pipe_kernel<T, -1><<<p.fft_grid[2], th, sm, s>>>(g, p.fyr, tsy, grid, p.zrange, lcw, kxs, kxe);
    else
      col_pipe_kernel<T, +1><<<p.fft_grid[3], th, sm, s>>>(g, p.fyr, tsy, grid, p.zrange, lcw, kxs, kxe);
    return;
  }
  if (p.fft_reg[1]) {
    const int th = reg_threads(p.fyr, lcw);
    const size_t sm = reg_smem<T>(g.ny << lcw);
    if (dir < 0)
      col_reg_kernel<T, -1><<<p.fft_grid[2], th, sm, s>>>(g, p.fyr, tsy, grid, p.zrange, lcw, kxs, kxe);
    else
      col_reg_kernel<T, +1><<<p.fft_grid[3], th, sm, s>>>(g, p.fyr, tsy, grid, p.zrange, lcw, kxs, kxe);
    return;
  }
  const size_t sm = col_smem<T>(g, lcw);
  const int th = fft_threads(g.ny << lcw);
  if (dir < 0)
    col_kernel<T, -1><<<p.fft_grid[2], th, sm, s>>>(g, p.fy, twy, reinterpret_cast<cplx<T>*>(p.grid), p.zrange, lcw,
                                                    kxs, kxe);
  else
    col_kernel<T, +1><<<p.fft_grid[3], th, sm, s>>>(g, p.fy, twy, reinterpret_cast<cplx<T>*>(p.grid), p.zrange, lcw,
                                                    kxs, kxe);
}

template int fft_smem_ok<float>(Plan&);
template int fft_smem_ok<double>(Plan&);
template int fft_set_row_variant<float>(Plan&, int);
template int fft_set_row_variant<double>(Plan&, int);
template int fft_set_col_width<float>(Plan&, int, int);
template int fft_set_col_width<double>(Plan&, int, int);
template void launch_fft_rows<float>(const Plan&, int, cudaStream_t);
template void launch_fft_rows<double>(const Plan&, int, cudaStream_t);
template void launch_fft_cols<float>(const Plan&, int, int, int, cudaStream_t);
template void launch_fft_cols<double>(const Plan&, int, int, int, cudaStream_t);

template <typename T>
int fft_col_width(const Plan& p) { return 1 << p.col_lcw; }
template int fft_col_width<float>(const Plan&);
template int fft_col_width<double>(const Plan&);

}  // namespace dps
