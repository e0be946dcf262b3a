// dpstokes_spread_noalloc: the spreading stage (particle records, binning, tile-gather spread) for
// callers that cannot allocate device memory.  Its scratch lives in one file-scope device array of
// fixed size that every GPU loading the library holds until the process exits; nothing here calls
// cudaMalloc, cudaFree or any allocating routine.
#include <math.h>
#include <string.h>

#include <algorithm>
#include <mutex>
#include <vector>

#include "dps_internal.cuh"

namespace dps {
namespace {

constexpr size_t kNoAllocScratchBytes = (size_t)64 << 20;  // 64 MiB per device

static __device__ __align__(256) unsigned char g_noalloc_scratch[kNoAllocScratchBytes];

// Host-side addresses of the array, one per device; filled on the first call made on that device.
constexpr int kMaxDevices = 64;
std::mutex g_addr_mutex;
void* g_addr[kMaxDevices] = {nullptr};

dps_status scratch_address(int dev, unsigned char** out) {
  if (dev < 0 || dev >= kMaxDevices) return DPS_ERR_INVALID_ARG;
  std::lock_guard<std::mutex> lock(g_addr_mutex);
  if (!g_addr[dev]) {
    void* ptr = nullptr;
    // the symbol's name is a host-side stand-in; only this call yields the device address
    if (cudaGetSymbolAddress(&ptr, g_noalloc_scratch) != cudaSuccess || !ptr) return DPS_ERR_CUDA;
    g_addr[dev] = ptr;
  }
  *out = reinterpret_cast<unsigned char*>(g_addr[dev]);
  return DPS_OK;
}

// Chebyshev node heights, computed on the host by the same expression as a plan's table and passed
// by value (2 KB of kernel parameters), so both paths place every envelope on identical nodes.
struct NodeTable {
  double z[257];
};

__global__ void noalloc_init_kernel(double* zc, const NodeTable nodes, int nz, int* zrange, int* status,
                                    int* bin_count, int nbins) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < nz) zc[i] = nodes.z[i];
  if (i == 0) {
    zrange[0] = nz;
    zrange[1] = -1;
    status[0] = 0;
  }
  for (int b = i; b < nbins; b += gridDim.x * blockDim.x) bin_count[b] = 0;
}

size_t align256(size_t x) { return (x + 255) / 256 * 256; }

}  // namespace
}  // namespace dps

extern "C" dps_status dpstokes_spread_noalloc(double Lx, double Ly, double zmin, double zmax, int32_t wall_mode,
                                              const dps_grid* grid, const dps_kernel_params* kp, int64_t n,
                                              const double* positions, const double* forces,
                                              const double* torques, double* out_grid, int64_t ldx,
                                              void* stream) {
  using namespace dps;
  if (!grid || !kp || n < 0 || !out_grid) return DPS_ERR_INVALID_ARG;
  if (!(Lx > 0) || !(Ly > 0) || !(zmax > zmin) || !isfinite(Lx) || !isfinite(Ly) || !isfinite(zmin) ||
      !isfinite(zmax))
    return DPS_ERR_INVALID_ARG;
  if (wall_mode < DPS_FREE || wall_mode > DPS_SLIT) return DPS_ERR_INVALID_ARG;
  const int nx = grid->nx, ny = grid->ny, nz = grid->nz;
  if (nx < 8 || ny < 8 || nz < 5 || nz > 257) return DPS_ERR_INVALID_ARG;
  if (ldx < nx || (ldx & 1)) return DPS_ERR_INVALID_ARG;
  const double hx = Lx / nx, hy = Ly / ny;
  if (fabs(hx - hy) > 1e-12 * hx) return DPS_ERR_INVALID_ARG;
  const bool torque = kp->with_torque != 0;
  if (n > 0 && (!positions || !forces || (torque && !torques))) return DPS_ERR_INVALID_ARG;
  if (!torque && torques) return DPS_ERR_INVALID_ARG;

  // geometry of the spreading stage, double precision, caller's row stride
  Plan p;
  memset(&p, 0, sizeof(Plan));
  Geometry& g = p.g;
  g.Lx = Lx; g.Ly = Ly; g.zmin = zmin; g.zmax = zmax; g.H = zmax - zmin; g.sH = 2.0 / g.H;
  g.h = hx; g.inv_h = 1.0 / hx; g.eta = 1.0; g.inv_eta = 1.0; g.mode = wall_mode;
  g.nx = nx; g.ny = ny; g.nz = nz; g.nkx = nx / 2 + 1;
  g.pitch = (int)(ldx / 2);  // the spreading kernel writes rows of 2 * pitch values
  if (particle_geometry(g, kp, 2) != DPS_OK) return DPS_ERR_INVALID_ARG;

  // carve the scratch: node table, plane range, status, bins, particle records
  const int nbins = g.nbx * g.nby;
  const size_t nn = (size_t)std::max<int64_t>(n, 1);
  size_t off = 0;
  const size_t o_zc = off; off = align256(off + (size_t)nz * sizeof(double));
  const size_t o_zr = off; off = align256(off + 2 * sizeof(int));
  const size_t o_st = off; off = align256(off + sizeof(int));
  const size_t o_bc = off; off = align256(off + (size_t)nbins * sizeof(int));
  const size_t o_bs = off; off = align256(off + (size_t)(nbins + 1) * sizeof(int));
  const size_t o_bu = off; off = align256(off + (size_t)nbins * sizeof(int));
  const size_t o_bo = off; off = align256(off + nn * sizeof(int));
  const size_t o_so = off; off = align256(off + nn * sizeof(int));
  const size_t o_rc = off; off = align256(off + nn * (size_t)g.rec_words * sizeof(uint32_t));
  if (off > kNoAllocScratchBytes) return DPS_ERR_INVALID_ARG;  // problem larger than the fixed scratch

  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return DPS_ERR_CUDA;
  unsigned char* base = nullptr;
  const dps_status st = scratch_address(dev, &base);
  if (st != DPS_OK) return st;
  p.device = dev;
  p.precision = DPS_FP64;
  p.max_n = n;
  p.tab.zc = reinterpret_cast<double*>(base + o_zc);
  p.zrange = reinterpret_cast<int*>(base + o_zr);
  p.status = reinterpret_cast<int*>(base + o_st);
  p.bin_count = reinterpret_cast<int*>(base + o_bc);
  p.bin_start = reinterpret_cast<int*>(base + o_bs);
  p.bin_cursor = reinterpret_cast<int*>(base + o_bu);
  p.bin_of = reinterpret_cast<int*>(base + o_bo);
  p.sorted = reinterpret_cast<int*>(base + o_so);
  p.records = reinterpret_cast<uint32_t*>(base + o_rc);
  p.grid = out_grid;

  cudaStream_t s = (cudaStream_t)stream;
  // every plane of the output starts at zero; the spread overwrites the occupied planes
  if (cudaMemsetAsync(out_grid, 0, (size_t)g.nfields * nz * ny * (size_t)ldx * sizeof(double), s) != cudaSuccess)
    return DPS_ERR_CUDA;
  const int blocks = std::min(1024, std::max(nz, nbins) / 256 + 1);
  NodeTable nodes;
  for (int c = 0; c < nz; ++c) nodes.z[c] = zmin + 0.5 * g.H * (1.0 + cos(M_PI * c / (nz - 1)));
  noalloc_init_kernel<<<blocks, 256, 0, s>>>(p.tab.zc, nodes, nz, p.zrange, p.status, p.bin_count, nbins);
  const int sp = spread_prepare<double>(p);
  if (sp < 0) return DPS_ERR_INVALID_ARG;
  if (sp == 0) return DPS_ERR_CUDA;
  launch_records<double>(p, n, positions, forces, torques, s);
  launch_bins(p, n, s);
  launch_spread<double>(p, s);
  return cudaGetLastError() == cudaSuccess ? DPS_OK : DPS_ERR_CUDA;
}
