// Conjugate-partner pairing of the register-staged row passes (plain C++, host and device).
//
// A real-data transform of n points packs two real rows as z = r0 + i r1; its half spectra need z_k
// together with z_{n-k}.  In a Stockham stage of radix R and span ns = n / R (the last stage of the
// forward pass, the first of the inverse), butterfly jj handles the values k = jj + ns r (r < R),
// and the partner n - k = (ns - jj) + ns (R - 1 - r) belongs to butterfly ns - jj.  Thread t of a
// stage with ns butterflies (ns a multiple of 32) takes butterfly pair_butterfly(t, ns): in warp w,
// lanes 0-15 take x = 16 w + lane and lanes 16-31 the partners ns - x, except that lane 16 of warp 0
// takes ns / 2 (butterflies 0 and ns / 2 are their own partners), so the partner of the butterfly
// of lane l sits in lane l ^ 16 of the same warp and a shuffle exchanges their values.
#pragma once

namespace dps {

#if defined(__CUDACC__)
#define DPS_HD __host__ __device__
#else
#define DPS_HD
#endif

DPS_HD inline int pair_butterfly(int t, int ns) {
  const int lane = t & 31, x = 16 * (t >> 5) + (lane & 15);
  return lane < 16 ? x : (x == 0 ? ns / 2 : ns - x);
}

// butterflies that are their own conjugate partners (they use their own values, not the shuffle's)
DPS_HD inline bool pair_self(int jj, int ns) { return jj == 0 || 2 * jj == ns; }

#undef DPS_HD

}  // namespace dps
