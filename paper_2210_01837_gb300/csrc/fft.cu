// In-house xy FFTs of the Chebyshev planes (steps 2 and 7 of Sec. III.D, xy part).
//
// Forward: f_hat(k) = sum_x f(x) exp(-i k.x) (unnormalised).  Inverse: sum_k f_hat(k) exp(+i k.x);
// the 1/(Nx Ny) factor is applied by the per-k solver when it writes its outputs.
//
// Layout of one field/plane: ny rows; each row holds nx reals in real space and nx/2+1 complex
// values (pitch >= nx/2+1 complex) in x-Fourier space, in place.
//   * row pass:    one block transforms two real rows packed as one complex sequence
//                  (z = r0 + i r1), then separates the two half spectra; inverse likewise.
//   * column pass: one block transforms `cw` adjacent x-wavenumber columns along y.
// Each 1D transform is a self-sorting (Stockham) mixed-radix FFT in shared memory written from the
// textbook formulation: stage s with radix R and span Ns multiplies input j + r n/R by
// W_{Ns R}^{(j mod Ns) r}, applies an R-point DFT, and stores to (j / Ns) Ns R + (j mod Ns) + r Ns.
// Radices 8, 4, 2 (hand-written butterflies) and 3, 5, 7 (direct DFT with exact constants).
// Twiddles W_n^t = exp(-2 pi i t/n) come from a table built in double precision on the host.
#include "dps_internal.cuh"

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

// Shared-memory index with one pad element per 16: breaks the power-of-two strides of the
// Stockham writes across bank groups.
__device__ __forceinline__ int pad16(int i) { return i + (i >> 4); }

// One Stockham stage over `batch` interleaved sequences (element e of sequence b at e*batch + b,
// batch a power of two given by its log).  Division by the span Ns uses a multiply-high with a
// per-stage magic number (exact for indices below 2^20).
template <typename T, int R, int DIR>
__device__ __forceinline__ void stage(const cplx<T>* __restrict__ in, cplx<T>* __restrict__ out, int n, int Ns,
                                      unsigned long long magic, int lbatch, const cplx<T>* __restrict__ tw) {
  const int nr = n / R;
  const int batch = 1 << lbatch;
  const int total = nr << lbatch;
  const int tstep = n / (Ns * R);
  for (int t = threadIdx.x; t < total; t += blockDim.x) {
    const int b = t & (batch - 1);
    const int jj = t >> lbatch;
    const int q = (int)(((unsigned long long)jj * magic) >> 40);
    const int k = jj - q * Ns;
    cplx<T> v[R];
#pragma unroll
    for (int r = 0; r < R; ++r) v[r] = in[pad16(((jj + r * nr) << lbatch) + b)];
    if (Ns > 1) {
#pragma unroll
      for (int r = 1; r < R; ++r) {
        cplx<T> w = tw[k * r * tstep];
        if (DIR > 0) w.y = -w.y;
        v[r] = v[r] * w;
      }
    }
    Dft<T, R, DIR>::run(v);
    const int base = q * Ns * R + k;
#pragma unroll
    for (int r = 0; r < R; ++r) out[pad16(((base + r * Ns) << lbatch) + b)] = v[r];
  }
}

// Full transform; returns the buffer that holds the result.
template <typename T, int DIR>
__device__ cplx<T>* fft_smem(cplx<T>* b0, cplx<T>* b1, const FftPlan& fp, int lbatch, const cplx<T>* tw) {
  int Ns = 1;
  cplx<T>* in = b0;
  cplx<T>* out = b1;
  for (int s = 0; s < fp.nstages; ++s) {
    const int R = fp.radix[s];
    const unsigned long long mg = fp.magic[s];
    switch (R) {
      case 16: stage<T, 16, DIR>(in, out, fp.n, Ns, mg, lbatch, tw); break;
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

__device__ __forceinline__ bool plane_live(const int* zrange, int c) { return c >= zrange[0] && c <= zrange[1]; }

template <typename T>
__global__ void row_r2c_kernel(Geometry g, FftPlan fp, const cplx<T>* __restrict__ tw, T* __restrict__ grid,
                               const int* __restrict__ zrange) {
  extern __shared__ __align__(16) unsigned char smraw[];
  cplx<T>* b0 = reinterpret_cast<cplx<T>*>(smraw);
  cplx<T>* b1 = b0 + pad16(g.nx);
  const int c = blockIdx.y, f = blockIdx.z;
  if (!plane_live(zrange, c)) return;
  const int y0 = 2 * blockIdx.x, y1 = y0 + 1;
  const bool has1 = y1 < g.ny;
  const size_t rowlen = (size_t)2 * g.pitch;
  T* row0 = grid + ((size_t)(f * g.nz + c) * g.ny + y0) * rowlen;
  T* row1 = row0 + rowlen;
  for (int a = threadIdx.x; a < g.nx; a += blockDim.x) b0[pad16(a)] = mk<T>(row0[a], has1 ? row1[a] : (T)0);
  __syncthreads();
  const cplx<T>* res = fft_smem<T, -1>(b0, b1, fp, 0, tw);
  cplx<T>* c0 = reinterpret_cast<cplx<T>*>(row0);
  cplx<T>* c1 = reinterpret_cast<cplx<T>*>(row1);
  const T half = (T)0.5;
  for (int k = threadIdx.x; k <= g.nx / 2; k += blockDim.x) {
    const cplx<T> zk = res[pad16(k)];
    const cplx<T> zm = conjg(res[pad16(k == 0 ? 0 : g.nx - k)]);
    c0[k] = scl(zk + zm, half);
    if (has1) {
      const cplx<T> d = zk - zm;  // (zk - conj z_{-k}) / (2i)
      c1[k] = mk<T>(half * d.y, -half * d.x);
    }
  }
}

template <typename T>
__global__ void row_c2r_kernel(Geometry g, FftPlan fp, const cplx<T>* __restrict__ tw, T* __restrict__ grid,
                               const int* __restrict__ zrange) {
  extern __shared__ __align__(16) unsigned char smraw[];
  cplx<T>* b0 = reinterpret_cast<cplx<T>*>(smraw);
  cplx<T>* b1 = b0 + pad16(g.nx);
  const int c = blockIdx.y, f = blockIdx.z;
  if (!plane_live(zrange, c)) return;
  const int y0 = 2 * blockIdx.x, y1 = y0 + 1;
  const bool has1 = y1 < g.ny;
  const size_t rowlen = (size_t)2 * g.pitch;
  T* row0 = grid + ((size_t)(f * g.nz + c) * g.ny + y0) * rowlen;
  T* row1 = row0 + rowlen;
  const cplx<T>* c0 = reinterpret_cast<const cplx<T>*>(row0);
  const cplx<T>* c1 = reinterpret_cast<const cplx<T>*>(row1);
  for (int k = threadIdx.x; k <= g.nx / 2; k += blockDim.x) {
    const cplx<T> x0 = c0[k];
    const cplx<T> x1 = has1 ? c1[k] : mk<T>((T)0, (T)0);
    b0[pad16(k)] = x0 + mul_i(x1);
    if (k > 0 && k < g.nx - k) b0[pad16(g.nx - k)] = conjg(x0) + mul_i(conjg(x1));
  }
  __syncthreads();
  const cplx<T>* res = fft_smem<T, +1>(b0, b1, fp, 0, tw);
  for (int a = threadIdx.x; a < g.nx; a += blockDim.x) {
    const cplx<T> v = res[pad16(a)];
    row0[a] = v.x;
    if (has1) row1[a] = v.y;
  }
}

template <typename T, int DIR>
__global__ void col_kernel(Geometry g, FftPlan fp, const cplx<T>* __restrict__ tw, cplx<T>* __restrict__ grid,
                           const int* __restrict__ zrange, int lcw, int kxs, int kxe) {
  extern __shared__ __align__(16) unsigned char smraw[];
  const int cw = 1 << lcw;
  cplx<T>* b0 = reinterpret_cast<cplx<T>*>(smraw);
  cplx<T>* b1 = b0 + pad16(g.ny * cw);
  const int c = blockIdx.y, f = blockIdx.z;
  if (!plane_live(zrange, c)) return;
  const int kx0 = kxs + blockIdx.x * cw;
  const int ncols = min(cw, kxe - kx0);
  cplx<T>* base = grid + (size_t)(f * g.nz + c) * g.ny * g.pitch + kx0;
  const int tot = g.ny << lcw;
  for (int t = threadIdx.x; t < tot; t += blockDim.x) {
    const int y = t >> lcw, b = t & (cw - 1);
    b0[pad16(t)] = (b < ncols) ? base[(size_t)y * g.pitch + b] : mk<T>((T)0, (T)0);
  }
  __syncthreads();
  const cplx<T>* res = fft_smem<T, DIR>(b0, b1, fp, lcw, tw);
  for (int t = threadIdx.x; t < tot; t += blockDim.x) {
    const int y = t >> lcw, b = t & (cw - 1);
    if (b < ncols) base[(size_t)y * g.pitch + b] = res[pad16(t)];
  }
}

size_t padded_bytes(int n, size_t esz) { return (size_t)(n + (n >> 4) + 1) * esz; }

// log2 of the column block: widest power of two (at most 8) whose two padded buffers leave room for
// two blocks per SM (100 KB each), else one block (200 KB)
template <typename T>
int col_lwidth(const Plan& p) {
  for (int l = 3; l > 0; --l)
    if (2 * padded_bytes(p.g.ny << l, sizeof(cplx<T>)) <= 100 * 1024) return l;
  for (int l = 3; l > 0; --l)
    if (2 * padded_bytes(p.g.ny << l, sizeof(cplx<T>)) <= 200 * 1024) return l;
  return 0;
}

}  // namespace

template <typename T>
int fft_smem_ok(const Plan& p) {
  const size_t row = 2 * padded_bytes(p.g.nx, sizeof(cplx<T>));
  const size_t col = 2 * padded_bytes(p.g.ny << col_lwidth<T>(p), sizeof(cplx<T>));
  if (row > 220 * 1024 || col > 220 * 1024) return 0;
  cudaFuncSetAttribute(row_r2c_kernel<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)row);
  cudaFuncSetAttribute(row_c2r_kernel<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)row);
  cudaFuncSetAttribute(col_kernel<T, -1>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)col);
  cudaFuncSetAttribute(col_kernel<T, +1>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)col);
  return 1;
}

template <typename T>
void launch_fft_rows(const Plan& p, int dir, cudaStream_t s) {
  const Geometry& g = p.g;
  const cplx<T>* twx = reinterpret_cast<const cplx<T>*>(p.tab.twx);
  dim3 gr((g.ny + 1) / 2, g.nz, g.nfields);
  const size_t sm = 2 * padded_bytes(g.nx, sizeof(cplx<T>));
  if (dir < 0)
    row_r2c_kernel<T><<<gr, 256, sm, s>>>(g, p.fx, twx, reinterpret_cast<T*>(p.grid), p.zrange);
  else
    row_c2r_kernel<T><<<gr, 256, sm, s>>>(g, p.fx, twx, reinterpret_cast<T*>(p.grid), p.zrange);
}

template <typename T>
void launch_fft_cols(const Plan& p, int dir, int kxs, int kxe, cudaStream_t s) {
  const Geometry& g = p.g;
  const cplx<T>* twy = reinterpret_cast<const cplx<T>*>(p.tab.twy);
  const int lcw = col_lwidth<T>(p);
  const int cw = 1 << lcw;
  dim3 gc((kxe - kxs + cw - 1) / cw, g.nz, g.nfields);
  const size_t sm = 2 * padded_bytes(g.ny << lcw, sizeof(cplx<T>));
  if (dir < 0)
    col_kernel<T, -1><<<gc, 512, sm, s>>>(g, p.fy, twy, reinterpret_cast<cplx<T>*>(p.grid), p.zrange, lcw, kxs, kxe);
  else
    col_kernel<T, +1><<<gc, 512, sm, s>>>(g, p.fy, twy, reinterpret_cast<cplx<T>*>(p.grid), p.zrange, lcw, kxs, kxe);
}

template int fft_smem_ok<float>(const Plan&);
template int fft_smem_ok<double>(const Plan&);
template void launch_fft_rows<float>(const Plan&, int, cudaStream_t);
template void launch_fft_rows<double>(const Plan&, int, cudaStream_t);
template void launch_fft_cols<float>(const Plan&, int, int, int, cudaStream_t);
template void launch_fft_cols<double>(const Plan&, int, int, int, cudaStream_t);

template <typename T>
int fft_col_width(const Plan& p) { return 1 << col_lwidth<T>(p); }
template int fft_col_width<float>(const Plan&);
template int fft_col_width<double>(const Plan&);

}  // namespace dps
