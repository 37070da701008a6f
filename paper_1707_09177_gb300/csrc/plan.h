// Host-side planning of the FFT passes, shared by every entry point that
// launches them (the context-owning solvers and the allocation-free filter):
// the radix decomposition of a transform length, the Stockham stage table,
// and the tile width / block size / shared-memory row stride of a pass. The
// pass kernels take their fixed-plan fast path only when a plan equals the
// compile-time plan for its length, so every launcher must build plans the
// same way; keeping one copy here guarantees that.
#pragma once

#include <cmath>
#include <cstddef>

#include "args.h"

namespace gad {

// Padded shared-memory index of element i (one pad slot every 16 elements).
inline int phys_h(int i) { return i + (i >> 4); }

inline bool smooth23(long long n) {
  if (n < 1) return false;
  while (n % 2 == 0) n /= 2;
  while (n % 3 == 0) n /= 3;
  return n == 1;
}

// Largest power of two dividing n (capped at 2^20).
inline int pow2_part(long long n) {
  int p = 1;
  while (n % 2 == 0 && p < (1 << 20)) { n /= 2; p *= 2; }
  return p;
}

// Elements per FFT thread: 24 when the length has a factor 3, else 16.
inline int pick_E(int L) { return (L % 3 == 0) ? 24 : 16; }

constexpr int kMaxStages = 5;       // the kernels unroll at most 5 stages

// Balanced radix list for a length L and E elements per thread: the factors 3
// first, then the power of two split into as few stages of at most 2^4 (E =
// 16) or 2^3 (E = 24) as possible, the larger radices first. Writes at most
// kMaxStages radices into rad and returns their number, or 0 when L is not
// 2^a 3^b, a radix does not divide E, or more stages would be needed.
inline int radices_for(int L, int E, int* rad) {
  int n = L, a = 0, b = 0;
  while (n > 1 && n % 2 == 0) { n /= 2; ++a; }
  while (n > 1 && n % 3 == 0) { n /= 3; ++b; }
  if (n != 1 || (a == 0 && b == 0)) return 0;
  if (b > 0 && E % 3 != 0) return 0;
  const int maxlog = (E % 16 == 0) ? 4 : 3;
  const int ns = a > 0 ? (a + maxlog - 1) / maxlog : 0;
  if (b + ns > kMaxStages) return 0;
  int k = 0;
  for (int i = 0; i < b; ++i) rad[k++] = 3;
  for (int i = 0; i < ns; ++i) rad[k++] = 1 << (a / ns + (i < a % ns ? 1 : 0));
  for (int i = 0; i < k; ++i)
    if (E % rad[i] != 0) return 0;
  return k;
}

// Stockham stage table for the radices rad[0..nrad) (in that order) over the
// plan's twiddle table `tab` (see FftPlan; fill it with plan_twiddles).
inline bool make_fft_from(int L, const int* rad, int nrad, const void* tab, FftPlan& fp) {
  if (nrad < 1 || nrad > kMaxStages) return false;
  fp = FftPlan{};
  fp.L = L;
  fp.nst = nrad;
  fp.tw = tab;
  long long ns = 1, off = 0;
  for (int q = 0; q < nrad; ++q) {
    FftStage& s = fp.st[q];
    s.radix = rad[q];
    s.ns = (int)ns;
    s.tw_off = (int)off;
    s.rcp_lr = 1.0f / (float)(L / rad[q]);
    s.rcp_ns = 1.0f / (float)ns;
    off += (long long)(rad[q] - 1) * ns;
    ns *= rad[q];
  }
  return ns == L;
}

// Radices of the plan of length L for E elements per thread; `reversed` gives
// them in reverse order (the filter pass's inverse transform, whose first
// stage meets the forward transform's last stage in registers). Returns the
// number of stages, 0 when there is no plan.
inline int plan_radices(int L, int E, bool reversed, int* rad) {
  const int n = radices_for(L, E, rad);
  if (reversed)
    for (int i = 0; i < n / 2; ++i) {
      const int t = rad[i];
      rad[i] = rad[n - 1 - i];
      rad[n - 1 - i] = t;
    }
  return n;
}

inline bool make_fft(int L, int E, const void* tab, FftPlan& fp, bool reversed = false) {
  int rad[kMaxStages];
  const int n = plan_radices(L, E, reversed, rad);
  return n > 0 && make_fft_from(L, rad, n, tab, fp);
}

// The plan's twiddle table (L - 1 complex entries, interleaved re, im) in
// long double, rounded to T: stage q, factor r, butterfly k at
// tw_off(q) + (r - 1) ns(q) + k holds exp(-2 pi i r k / (rad[q] ns(q))); the
// quarter and half turns are exact.
template <typename T>
inline void plan_twiddles(const int* rad, int nrad, T* out) {
  const long double two_pi = 6.283185307179586476925286766559005768L;
  long long ns = 1, off = 0;
  for (int q = 0; q < nrad; ++q) {
    const long long len = (long long)rad[q] * ns;
    for (int r = 1; r < rad[q]; ++r)
      for (long long k = 0; k < ns; ++k) {
        const long long m = ((long long)r * k) % len;
        long double c, sn;
        if (m == 0) { c = 1; sn = 0; }
        else if (4 * m == len) { c = 0; sn = -1; }
        else if (2 * m == len) { c = -1; sn = 0; }
        else if (4 * m == 3 * len) { c = 0; sn = 1; }
        else {
          const long double ang = two_pi * (long double)m / (long double)len;
          c = cosl(ang);
          sn = -sinl(ang);
        }
        const long long e = off + (long long)(r - 1) * ns + k;
        out[2 * e] = (T)c;
        out[2 * e + 1] = (T)sn;
      }
    off += (long long)(rad[q] - 1) * ns;
    ns *= rad[q];
  }
}

// Odd shared-memory row stride (complex units) of a tile row of `slots`
// elements.
inline int tile_ld(int slots) {
  int ld = phys_h(slots - 1) + 1;
  if ((ld & 1) == 0) ++ld;
  return ld;
}

struct TileShape {
  int E = 0, W = 0, T = 0, ld = 0;
  size_t smem = 0;
};

// Picks the tile width W (a power of two dividing `div`, or any power of two
// when div = 0) whose block size T = W*L/E is closest to 256 threads, with at
// most 100 KB of shared memory (rows of `slots` elements of csize bytes).
inline bool choose_tile(int L, int E, int slots, int div, size_t csize, TileShape& ts) {
  const int ld = tile_ld(slots);
  int bestW = 0, bestT = 0;
  double bestScore = 1e30;
  for (int W = 1; W <= 4096; W *= 2) {
    if (div > 0 && div % W != 0) break;
    const long long tot = (long long)W * L;
    if (tot % E != 0) continue;
    const long long T = tot / E;
    if (T < 1 || T > 256) continue;
    const size_t smem = (size_t)W * ld * csize;
    if (smem > 100 * 1024) continue;
    const double score = std::fabs(std::log2((double)T / 256.0));
    if (score < bestScore - 1e-9) { bestScore = score; bestW = W; bestT = (int)T; }
  }
  if (!bestW) return false;
  ts.E = E;
  ts.W = bestW;
  ts.T = bestT;
  ts.ld = ld;
  ts.smem = (size_t)bestW * ld * csize;
  return true;
}

}  // namespace gad
