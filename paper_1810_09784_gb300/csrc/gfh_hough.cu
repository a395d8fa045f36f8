// Generalized FrequencyHough accumulation (Sec. IV) on sm_103a.
//
// Each peak (FFT i, bin j) is the set of lines x0 = x - (n-1) k t_i for x across its bin
// (Eq. transform, Sec. IV).  On k row r it covers the x0 columns that the half-open fixed-point
// interval [U[j+1] - B_i - r S_i, U[j] - B_i - r S_i) overlaps.  The map is built per tile of
// R rows x C columns in shared memory by differential counting: +1 at the first covered column,
// -1 after the last (warp-level shared-memory atomics; intervals that start left of the tile go to
// a per-thread register carry instead of contending on column 0), then a running sum along x0 and
// one vectorised streaming store of every map cell.  Candidate selection (Sec. IV: highest count
// per f0 band, critical ratio from the map's mean and deviation) is fused into the store pass.
#include <cstdio>

#include "gfh_internal.h"

namespace {

constexpr int kLane = 32;

__device__ __forceinline__ int warp_sum(int v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

__device__ __forceinline__ long long warp_sum64(long long v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

__device__ __forceinline__ int warp_incl_scan(int v, int lane) {
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const int u = __shfl_up_sync(0xffffffffu, v, o);
    if (lane >= o) v += u;
  }
  return v;
}

// Candidate key: count in the high word, inverted row-major cell index in the low word, so the
// maximum key is the highest count with ties to the lowest (row, column).
__device__ __forceinline__ unsigned long long cand_key(int count, uint32_t lin) {
  return ((unsigned long long)(uint32_t)count << 32) | (unsigned long long)(0xffffffffu - lin);
}

// ---- per-execute preparation --------------------------------------------------------------------

// Flags peak lists whose bins are not sorted ascending.  fft_unsorted (may be null; n_flags
// entries, zeroed before): 1 for a list in which some bin's peaks are not in FFT order (the
// coarse-tile search then walks that list's peaks in full).
__global__ void k_check_sorted(const uint32_t* __restrict__ bins, const uint32_t* __restrict__ fft,
                               const int64_t* __restrict__ off, unsigned int* flag,
                               int* __restrict__ fft_unsorted, int n_flags) {
  const int l = blockIdx.y;
  const int64_t b = off[l], e = off[l + 1];
  const bool check_fft = fft_unsorted && l < n_flags;
  for (int64_t p = b + 1 + blockIdx.x * (int64_t)blockDim.x + threadIdx.x; p < e;
       p += (int64_t)gridDim.x * blockDim.x) {
    const uint32_t j1 = bins[p], j0 = bins[p - 1];
    if (j1 < j0) atomicOr(flag, GFH_FLAG_UNSORTED);
    else if (check_fft && j1 == j0 && fft[p] < fft[p - 1]) fft_unsorted[l] = 1;
  }
}

// Per map (blockIdx.y), bin jl and FFT block b: the offset in the bin's peaks of its first peak
// with FFT index >= kFftBlock b (the bin's count when none), by bisection over the bin's FFT
// indices.  Meaningful for lists whose bins hold their peaks in FFT order.
__global__ void k_fft_blocks(const MapDev* __restrict__ maps, const CoarseMapDev* __restrict__ cmaps,
                             const uint32_t* __restrict__ fft) {
  const MapDev& md = maps[blockIdx.y];
  const CoarseMapDev& cm = cmaps[blockIdx.y];
  const int J = md.bin_hi - md.bin_lo + 1;
  const int e = blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= J * cm.nb1) return;
  const int jl = e / cm.nb1, b = e - jl * cm.nb1;
  const int64_t s = md.csr[jl], t = md.csr[jl + 1];
  const uint32_t key = (uint32_t)b * (uint32_t)kFftBlock;
  int64_t lo = s, hi = t;
  while (lo < hi) {
    const int64_t mid = lo + ((hi - lo) >> 1);
    if (__ldg(fft + mid) < key) lo = mid + 1; else hi = mid;
  }
  cm.fblk[e] = (int32_t)(lo - s);
}

// csr[e] = index of the first peak of the map's list whose bin is >= bin_lo + e.
__global__ void k_csr(const MapDev* __restrict__ maps, const int32_t* __restrict__ entry_map,
                      int n_entries, const uint32_t* __restrict__ bins,
                      const int64_t* __restrict__ off) {
  const int q = blockIdx.x * blockDim.x + threadIdx.x;
  if (q >= n_entries) return;
  const MapDev& md = maps[entry_map[q]];
  const int e = q - md.csr_base;
  const uint32_t key = (uint32_t)(md.bin_lo + e);
  int64_t lo = off[md.list], hi = off[md.list + 1];
  while (lo < hi) {
    const int64_t mid = lo + ((hi - lo) >> 1);
    if (bins[mid] < key) lo = mid + 1; else hi = mid;
  }
  md.csr[e] = lo;
}

__global__ void k_set_offsets(int64_t* off, int64_t n) {
  if (threadIdx.x == 0) { off[0] = 0; off[1] = n; }
}

// Table rows of peak (f, bin): the FFT's base and shift per row, the bin's fixed-point edges.
// Returns false (and flags the input) for an out-of-range FFT index or a bin outside the map band,
// which only an unsorted peak list can put in a tile's range; the rows are then not read.
__device__ __forceinline__ bool peak_rows(const longlong2* __restrict__ BS,
                                          const longlong2* __restrict__ UP, int bin_lo, uint32_t f,
                                          int bin, uint32_t nfft, unsigned jmax,
                                          unsigned int* flag, longlong2& bs, longlong2& up) {
  const unsigned jl = (unsigned)(bin - bin_lo);
  if (f >= nfft) { atomicOr(flag, GFH_FLAG_FFT_RANGE); return false; }
  if (jl > jmax) { atomicOr(flag, GFH_FLAG_UNSORTED); return false; }
  bs = __ldg(BS + f);
  up = __ldg(UP + jl);
  return true;
}

// Interval of a peak on the tile's first row from its table rows: [A, B1 + 1) in 2^-32 columns,
// and its per-row shift S.
__device__ __forceinline__ void peak_interval(int row0, const longlong2 bs, const longlong2 up,
                                              int64_t& A, int64_t& B1, int64_t& S) {
  S = bs.y;
  const int64_t base = bs.x + (int64_t)row0 * S;
  A = up.x - base;        // interval start (upper-f edge)
  B1 = up.y - base - 1;   // interval end - 1 (lower-f edge)
}


// Whether the interval of a peak ([a, b1 + 1) on the tile's first row, shifted left by s >= 0 per
// row: t_first >= 0 and dk > 0 make every S_i non-negative) meets columns c0 .. ub on any of the
// R rows: its right edge is highest on the first row and its left edge lowest on the last.  A
// tile's bin range holds every bin that some FFT can bring into the tile at some row, so on a tall
// map many of the peaks read lie outside it on all R rows; they draw nothing and are skipped whole.
template <int R>
__device__ __forceinline__ bool meets_tile(int64_t a, int64_t b1, int64_t s, int c0, int ub) {
  return (b1 >> GFH_FRAC_BITS) >= (int64_t)c0 &&
         ((a - (int64_t)(R - 1) * s) >> GFH_FRAC_BITS) <= (int64_t)ub;
}

// Largest i in [-1, n) with shift B_i + r S_i <= x on row r; with k_min >= 0 the shift does not
// fall as i grows (t_i grows, dk > 0).  The guess comes from the straight line through the
// table's first and last rows (B_i and S_i are floors of linear functions of t_i, so it is off by
// far less than one FFT); the table confirms it with two loads issued together, and a bisection
// over the table settles a guess it does not confirm.
__device__ __forceinline__ int last_shift_at_most(const longlong2* __restrict__ BS, int n,
                                                  int64_t r, int64_t x, int64_t base0,
                                                  double inv_slope) {
  int i;
  if (inv_slope > 0.0) {
    const double e = floor((double)(x - base0) * inv_slope);
    i = e < -1.0 ? -1 : (e > (double)(n - 1) ? n - 1 : (int)e);
  } else {
    i = x >= base0 ? n - 1 : -1;        // every row of the table holds the same shift
  }
  const longlong2 a = __ldg(BS + max(i, 0));
  const longlong2 b = __ldg(BS + min(i + 1, n - 1));
  if ((i < 0 || a.x + r * a.y <= x) && (i + 1 >= n || b.x + r * b.y > x)) return i;
  int lo = 0, hi = n;                   // count of the FFTs with shift <= x
  while (lo < hi) {
    const int mid = (lo + hi) >> 1;
    const longlong2 bs = __ldg(BS + mid);
    if (bs.x + r * bs.y <= x) lo = mid + 1; else hi = mid;
  }
  return lo - 1;
}

// Events of one peak on the R rows of a tile (layout described at k_hough below).  The interval
// on row 0 is [a, b1 + 1) in 2^-32 columns and moves left by s per row.  G0 + m is column m of row
// 0 in absolute column numbering (the tile's first column is c0); ub = min(last column of the
// tile, last column of the map).
// A peak that moves less than a column per row, starts at least R - 1 columns right of the tile's
// first column and ends before the tile's last column and inside the map stays clear of every
// edge on all R rows (its left edge is lowest on the last row, its right edge highest on row 0):
// no clamp, no carry, and on rows r > 0 a column is entered where the left edge moved and left
// where the right edge moved.
template <int R>
__device__ __forceinline__ bool peak_interior(int64_t a, int64_t b1, int64_t s, int c0, int c1m1,
                                              int ub) {
  constexpr int64_t kOne = int64_t(1) << GFH_FRAC_BITS;
  const int lo = (int)(a >> GFH_FRAC_BITS), hr = (int)(b1 >> GFH_FRAC_BITS);
  return (s < kOne) & (lo >= c0 + (R - 1)) & (hr <= ub) & (hr < c1m1) & (a <= b1);
}

// interior: draw in the interior form (the caller has checked peak_interior for this peak); the
// edge-following form below draws every peak, interior ones with the same events.
template <int R>
__device__ __forceinline__ void draw_peak(int* G0, int lds, int64_t a, int64_t b1, int64_t s,
                                          int c0, int c1m1, int ub, int& carry, bool interior) {
  constexpr int64_t kOne = int64_t(1) << GFH_FRAC_BITS;
  int lo = (int)(a >> GFH_FRAC_BITS);
  const int hr = (int)(b1 >> GFH_FRAC_BITS);    // row-0 last column before any clamp
  if (interior) {
    atomicAdd(G0 + lo, 1);
    atomicAdd(G0 + hr + 1, -1);
    int o1 = lo, o2 = hr;
#pragma unroll
    for (int rr = 1; rr < R; ++rr) {
      a -= s;
      b1 -= s;
      const int n1 = (int)(a >> GFH_FRAC_BITS), n2 = (int)(b1 >> GFH_FRAC_BITS);
      int* const Gr = G0 + rr * lds;
      if (n1 < o1) atomicAdd(Gr + n1, 1);
      if (n2 < o2) atomicAdd(Gr + o2, -1);
      o1 = n1;
      o2 = n2;
    }
    return;
  }
  // row 0: first / last covered column, clamped to the map's last column and to the tile
  int hi = min(hr, ub);
  int o1 = max(lo, c0), o2 = hi;
  if (o1 <= o2) {
    if (lo < c0) carry += 1;
    else atomicAdd(G0 + o1, 1);
    if (hi < c1m1) atomicAdd(G0 + hi + 1, -1);
  }
  // rows 1 .. R-1 (rows past the map's last k row are drawn too: they exist in shared memory
  // and are never stored).  A shift below one column per row moves each edge by at most one
  // column per row: the left edge enters column n1 when it moves, the right edge leaves column
  // o2 when it moves.  Edges are followed unclamped and an event is drawn only inside the tile's
  // columns: an event right of the map's last column (inside the last tile of a map) lands in a
  // cell that is never stored and changes no stored cell, because sums run rightwards and down.
  if (s < kOne) {
    o1 = lo;
    o2 = hr;
#pragma unroll
    for (int rr = 1; rr < R; ++rr) {
      a -= s;
      b1 -= s;
      const int n1 = (int)(a >> GFH_FRAC_BITS), n2 = (int)(b1 >> GFH_FRAC_BITS);
      int* const Gr = G0 + rr * lds;
      if ((n1 < o1) & ((unsigned)(n1 - c0) <= (unsigned)(c1m1 - c0))) atomicAdd(Gr + n1, 1);
      if ((n2 < o2) & ((unsigned)(o2 - c0) <= (unsigned)(c1m1 - c0))) atomicAdd(Gr + o2, -1);
      o1 = n1;
      o2 = n2;
    }
  } else {
    for (int rr = 1; rr < R; ++rr) {
      a -= s;
      b1 -= s;
      lo = (int)(a >> GFH_FRAC_BITS);
      const int n1 = max(lo, c0), n2 = min((int)(b1 >> GFH_FRAC_BITS), ub);
      int* const Gr = G0 + rr * lds;
      const int e2 = min(n2, o1 - 1);
      for (int m = n1; m <= e2; ++m) atomicAdd(Gr + m, 1);
      for (int m = max(o1, n2 + 1); m <= o2; ++m) atomicAdd(Gr + m, -1);
      o1 = n1;
      o2 = n2;
    }
  }
}

// Events of one peak on the R rows of a tile in the x-direction form: every row differenced along
// x0 (+1 at its first column, -1 after its last), so a row costs two events whatever the shift per
// row; an interval entering from the left of the tile counts in that row's carry.
template <int R>
__device__ __forceinline__ void draw_peak_x(int* G0, int lds, int64_t a, int64_t b1, int64_t s,
                                            int c0, int c1m1, int ub, int (&carry)[R]) {
#pragma unroll
  for (int rr = 0; rr < R; ++rr) {
    const int lo = (int)(a >> GFH_FRAC_BITS);
    const int hi = min((int)(b1 >> GFH_FRAC_BITS), ub);
    const int o1 = max(lo, c0);
    int* const Gr = G0 + rr * lds;
    if (o1 <= hi) {
      if (lo < c0) carry[rr] += 1;
      else atomicAdd(Gr + o1, 1);
      if (hi < c1m1) atomicAdd(Gr + hi + 1, -1);
    }
    a -= s;
    b1 -= s;
  }
}

// ---- the accumulation + running sums + select kernel --------------------------------------------

// A tile is R k rows x C columns.  Lane l draws its own peaks on all R rows.
//
// Shared memory holds G[R][C+2] int32, a mixed differential of the tile:
//   row 0:     along x0 - +1 at the first column an interval covers, -1 after its last, so that
//              M[0][m] = sum_{m' <= m} G[0][m'];
//   row r > 0: along k - +1 at each column the interval newly covers on row r, -1 at each column it
//              covered on row r-1 but no longer does, so that M[r][m] = M[r-1][m] + G[r][m].
// Along k a peak's interval shifts left by S_i < 1 column per row with the default k step, so on
// most rows it enters no column and leaves none: rows after the first cost about one event per
// (peak, row) instead of two.  Intervals are clamped to the tile and to the map's last column;
// an interval entering from the left of the tile on row 0 is a per-thread carry into column c0.
//
// Shared memory: G[R][C+2] | tot[32] row-0 chunk sums | skey[bands] candidate keys.
// XD (maps whose line moves more than two x0 columns per k row): every row differenced along x0
// and scanned on its own; chunk sums tot[R][32].
//
// SUB (the coarse-tile search): a tile flagged `sub` whose list holds each bin's peaks in FFT
// order walks only, per read bin, the peaks of the FFTs whose interval can meet it.  On a narrow
// tile over k rows where the FFTs' shifts spread far wider than the tile, most peaks of its bins
// miss it.  Each bin's window of FFTs comes from the shift table (last_shift_at_most), its peaks
// from the FFT-block index (whole 64-FFT blocks, so a few peaks outside the window are read and
// dropped by the meets test).  The bins' start offsets and a prefix sum of their counts take the
// last 8 sub_cap + 16 bytes of the dynamic shared memory.
template <int R, int NT, bool SELECT, bool XD = false, int LDS = 0, bool UNIF = false,
          bool SUB = false>
__device__ __forceinline__ void hough_tile(const MapDev* __restrict__ maps, const TileDev t,
                                           const uint32_t* __restrict__ fft_idx,
                                           const uint32_t* __restrict__ bins,
                                           unsigned int* __restrict__ flag, int c_max,
                                           unsigned char* smem,
                                           const CoarseMapDev* __restrict__ cmaps = nullptr,
                                           const int* __restrict__ fft_unsorted = nullptr,
                                           int sub_cap = 0) {
  constexpr int NW = NT / kLane;
  const MapDev& md = maps[t.map];
  const int C = t.ncols;
  // row stride: the plan's tile width + 2 when fixed at compile time (row offsets become
  // immediates), else this tile's
  const int lds = LDS ? LDS : C + 2;
  int* G = reinterpret_cast<int*>(smem);
  int* tot = G + R * (c_max + 2);
  unsigned long long* skey = reinterpret_cast<unsigned long long*>(tot + (XD ? R : 1) * kLane);
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int nb_tile = t.band_hi >= t.band_lo ? t.band_hi - t.band_lo + 1 : 0;
  const int c0 = (int)t.col0;
  const int c1m1 = c0 + C - 1;                   // last column of the tile
  const int ub = min(c1m1, (int)md.W - 1);       // ... and of the map
  const int nbw = t.bin_b - t.bin_a + 1;         // bins read
  bool use_sub = false;
  int* sub_pre = nullptr;                        // per read bin: first walk index (then the total)
  int* sub_st = nullptr;                         // per read bin: its first peak, from the tile's
  if constexpr (SUB) {
    use_sub = t.sub != 0 && nbw > 0 && nbw <= sub_cap && fft_unsorted[cmaps[t.map].list] == 0;
    uint32_t dyn_bytes;
    asm("mov.u32 %0, %%dynamic_smem_size;" : "=r"(dyn_bytes));
    sub_pre = reinterpret_cast<int*>(smem + dyn_bytes - (8u * (uint32_t)sub_cap + 16u));
    sub_st = sub_pre + sub_cap + 2;
  }

  for (int i = tid; i < R * lds / 2; i += NT) reinterpret_cast<int2*>(G)[i] = make_int2(0, 0);
  if (SELECT)
    for (int i = tid; i < nb_tile; i += NT) skey[i] = 0ull;
  if constexpr (SUB) {
    if (use_sub) {
      // per read bin: its window of FFTs, then its peaks in those FFTs' blocks
      const CoarseMapDev& cm = cmaps[t.map];
      const int64_t pb0 = md.csr[t.bin_a - md.bin_lo];
      const int64_t r0 = t.row0, r1 = (int64_t)t.row0 + (R - 1);
      const double sl0 = cm.db + (double)r0 * cm.ds, sl1 = cm.db + (double)r1 * cm.ds;
      const double inv0 = sl0 > 0.0 ? 1.0 / sl0 : 0.0, inv1 = sl1 > 0.0 ? 1.0 / sl1 : 0.0;
      for (int q = tid; q < nbw; q += NT) {
        const int jl = t.bin_a - md.bin_lo + q;
        const longlong2 up = __ldg(md.UP + jl);
        // right edge on the first row reaches c0; left edge on the last row stays left of ub + 1
        const int last = last_shift_at_most(md.BS, md.n_fft, r0,
                                            up.y - 1 - ((int64_t)c0 << GFH_FRAC_BITS),
                                            cm.b0 + r0 * cm.s0, inv0);
        const int first = last_shift_at_most(md.BS, md.n_fft, r1,
                                             up.x - ((int64_t)(ub + 1) << GFH_FRAC_BITS),
                                             cm.b0 + r1 * cm.s0, inv1) + 1;
        int st = 0, cnt = 0;
        if (first <= last) {
          const int32_t* fb = cm.fblk + (int64_t)jl * cm.nb1;
          const int o0 = fb[first / kFftBlock], o1 = fb[last / kFftBlock + 1];
          st = (int)(md.csr[jl] - pb0) + o0;
          cnt = o1 - o0;
        }
        sub_st[q] = st;
        sub_pre[q] = cnt;
      }
    }
  }
  __syncthreads();
  if constexpr (SUB) {
    if (use_sub) {
      // exclusive prefix of the counts (warp 0, 32 consecutive runs), the total after them
      if (warp == 0) {
        const int per = (nbw + kLane - 1) / kLane;
        const int q0 = min(lane * per, nbw), q1 = min(q0 + per, nbw);
        int sum = 0;
        for (int q = q0; q < q1; ++q) sum += sub_pre[q];
        const int incl = warp_incl_scan(sum, lane);
        int run = incl - sum;
        for (int q = q0; q < q1; ++q) {
          const int c = sub_pre[q];
          sub_pre[q] = run;
          run += c;
        }
        if (lane == kLane - 1) sub_pre[nbw] = incl;
      }
      __syncthreads();
    }
  }

  // ---- accumulate
  if (t.bin_a <= t.bin_b) {
    const int64_t pb = md.csr[t.bin_a - md.bin_lo];
    const int64_t pe = md.csr[t.bin_b - md.bin_lo + 1];
    const uint32_t nfft = (uint32_t)md.n_fft;
    const unsigned jmax = (unsigned)(md.bin_hi - md.bin_lo);
    const int bin_lo = md.bin_lo;                // map fields read once, kept in registers
    const longlong2* const BS = md.BS;
    const longlong2* const UP = md.UP;
    int* const G0 = G - c0;                      // rows indexed by absolute column
    int carry = 0;
    int carry_x[XD ? R : 1] = {};
    // Software pipeline over this thread's peaks p, p + NT, ...: the indices are loaded two
    // peaks ahead and the table rows one peak ahead of the peak being drawn; the next peak's
    // interval is formed from its rows after the current peak is drawn, so the loads have the
    // whole drawing to arrive.
    // this tile's peaks with 32-bit offsets (a range beyond 2^31 - 2^20 peaks raises the capacity
    // flag and is not drawn)
    const bool fits = pe - pb <= (int64_t)0x7fffffff - (1 << 20);
    if (!fits && tid == 0) atomicOr(flag, GFH_FLAG_CAPACITY);
    const uint32_t* const fl = fft_idx + pb;
    const uint32_t* const bl = bins + pb;
    const int np = fits ? (int)(pe - pb) : 0;
    // walk n peaks; fetch(i, f, j) gives the FFT and bin of the i-th (i < n)
    auto walk = [&](int n, auto fetch) {
      int p = tid;
      uint32_t f_nx = 0xffffffffu;               // indices of peak p + NT
      int j_nx = 0;
      int64_t a_cu = 0, b_cu = 0, s_cu = 0;      // interval of peak p
      bool ok_cu = false;
      if (p < n) {
        uint32_t f;
        int j;
        fetch(p, f, j);
        longlong2 bs, up;
        ok_cu = peak_rows(BS, UP, bin_lo, f, j, nfft, jmax, flag, bs, up);
        if (ok_cu) peak_interval(t.row0, bs, up, a_cu, b_cu, s_cu);
      }
      if (p + NT < n) fetch(p + NT, f_nx, j_nx);
      for (; p < n; p += NT) {
        uint32_t f_nn = 0xffffffffu;             // indices of peak p + 2 NT
        int j_nn = 0;
        if (p + 2 * NT < n) fetch(p + 2 * NT, f_nn, j_nn);
        longlong2 bs_nx = make_longlong2(0, 0), up_nx = make_longlong2(0, 0);
        const bool ok_nx = f_nx != 0xffffffffu &&
                           peak_rows(BS, UP, bin_lo, f_nx, j_nx, nfft, jmax, flag, bs_nx, up_nx);
        const bool draw = ok_cu && meets_tile<R>(a_cu, b_cu, s_cu, c0, ub);
        if constexpr (XD) {
          if (draw) draw_peak_x<R>(G0, lds, a_cu, b_cu, s_cu, c0, c1m1, ub, carry_x);
        } else if constexpr (UNIF) {
          // one drawing form per warp: the interior form when every drawing lane's peak is
          // interior, else the edge-following form for all, so that a warp never runs both
          const bool interior = __all_sync(__activemask(),
                                           !draw || peak_interior<R>(a_cu, b_cu, s_cu, c0, c1m1, ub));
          if (draw) draw_peak<R>(G0, lds, a_cu, b_cu, s_cu, c0, c1m1, ub, carry, interior);
        } else {
          if (draw)
            draw_peak<R>(G0, lds, a_cu, b_cu, s_cu, c0, c1m1, ub, carry,
                         peak_interior<R>(a_cu, b_cu, s_cu, c0, c1m1, ub));
        }
        peak_interval(t.row0, bs_nx, up_nx, a_cu, b_cu, s_cu);
        ok_cu = ok_nx;
        f_nx = f_nn; j_nx = j_nn;
      }
    };
    if (SUB && use_sub) {
      // walk index v: its bin q is the last with sub_pre[q] <= v (empty bins share the prefix of
      // the next), its peak the bin's first peak + v - sub_pre[q]
      const int n_sub = fits ? sub_pre[nbw] : 0;
      walk(n_sub, [&](int v, uint32_t& f, int& j) {
        int lo = 0, hi = nbw - 1;
        while (lo < hi) {
          const int mid = (lo + hi + 1) >> 1;
          if (sub_pre[mid] <= v) lo = mid; else hi = mid - 1;
        }
        f = __ldg(fl + sub_st[lo] + (v - sub_pre[lo]));
        j = t.bin_a + lo;
      });
    } else {
      walk(np, [&](int p, uint32_t& f, int& j) {
        f = __ldg(fl + p);
        j = (int)__ldg(bl + p);
      });
    }
    if constexpr (XD) {
#pragma unroll
      for (int rr = 0; rr < (XD ? R : 1); ++rr) {
        const int v = warp_sum(carry_x[rr]);
        if (lane == 0 && v) atomicAdd(G + rr * lds, v);
      }
    } else {
      const int v = warp_sum(carry);
      if (lane == 0 && v) atomicAdd(G, v);
    }
  }
  __syncthreads();

  // ---- row-0 chunk sums: chunk = 128 columns (32 lanes x 4); warp w owns chunks w, w+NW, ...
  const int nch = (C + 127) / 128;
  const int nsum = XD ? t.nrows * nch : nch;     // (row, chunk) sums: row 0 only, or every row
  for (int idx = warp; idx < nsum; idx += NW) {
    const int rr = idx / nch, ch = idx - rr * nch;
    const int col = ch * 128 + lane * 4;
    int s = 0;
    if (col < C) {
      const int2 u = *reinterpret_cast<const int2*>(&G[rr * lds + col]);
      const int2 w = *reinterpret_cast<const int2*>(&G[rr * lds + col + 2]);
      s = u.x + u.y + w.x + w.y;
    }
    s = warp_sum(s);
    if (lane == 0) tot[rr * kLane + ch] = s;
  }
  __syncthreads();

  // ---- row 0: running sum along x0; rows r > 0: running sum along k; store; candidates
  long long s1 = 0, s2 = 0;
  const uint32_t W32 = (uint32_t)md.W;
  // map fields of the store pass read once (a global store could otherwise force a reload)
  int32_t* const out = md.out + t.col0;
  const int64_t ld_out = md.ld;
  const int32_t* const col_band = md.col_band + t.col0;
  for (int ch = warp; ch < nch; ch += NW) {
    const int col = ch * 128 + lane * 4;
    const bool in = col < C;
    int band[4] = {-1, -1, -1, -1};
    // per column: best count over the rows so far and its row (strictly greater, so the first
    // row reaching the best count wins: the lowest cell index)
    int bc[4] = {-1, -1, -1, -1}, br[4] = {0, 0, 0, 0};
    if (SELECT && in) {
      const int4 bv = __ldg(reinterpret_cast<const int4*>(col_band + col));
      band[0] = bv.x; band[1] = bv.y; band[2] = bv.z; band[3] = bv.w;
    }
    const int cin = XD ? 0 : warp_sum((lane < ch) ? tot[lane] : 0);
    int4 v = make_int4(0, 0, 0, 0);
    for (int rr = 0; rr < t.nrows; ++rr) {
      int4 g = make_int4(0, 0, 0, 0);
      if (in) {
        const int2 u = *reinterpret_cast<const int2*>(&G[rr * lds + col]);
        const int2 w = *reinterpret_cast<const int2*>(&G[rr * lds + col + 2]);
        g = make_int4(u.x, u.y, w.x, w.y);
      }
      if (XD || rr == 0) {
        const int cr = XD ? warp_sum((lane < ch) ? tot[rr * kLane + lane] : 0) : cin;
        g.y += g.x; g.z += g.y; g.w += g.z;
        const int incl = warp_incl_scan(g.w, lane);
        const int add = cr + incl - g.w;
        v = make_int4(g.x + add, g.y + add, g.z + add, g.w + add);
      } else {
        v.x += g.x; v.y += g.y; v.z += g.z; v.w += g.w;
      }
      if (in) {
        const int64_t row = t.row0 + rr;
        __stcs(reinterpret_cast<int4*>(out + row * ld_out + col), v);
        if (SELECT) {
          const int vals[4] = {v.x, v.y, v.z, v.w};
#pragma unroll
          for (int q = 0; q < 4; ++q) {
            if (band[q] >= 0) {
              s1 += vals[q];
              s2 += (long long)vals[q] * vals[q];
              if (vals[q] > bc[q]) { bc[q] = vals[q]; br[q] = rr; }
            }
          }
        }
      }
    }
    if (SELECT) {
      unsigned long long best[4];
#pragma unroll
      for (int q = 0; q < 4; ++q)
        best[q] = cand_key(bc[q], (uint32_t)(t.row0 + br[q]) * W32 + (uint32_t)(t.col0 + col + q));
      // merge equal-band neighbours among the lane's 4 columns, then one shared atomic per run
      // (at the run's last column; every index static, so the arrays stay in registers)
      unsigned long long run = 0;
#pragma unroll
      for (int q = 0; q < 4; ++q) {
        run = (q > 0 && band[q] == band[q - 1]) ? (best[q] > run ? best[q] : run) : best[q];
        const bool last = q == 3 || band[q < 3 ? q + 1 : q] != band[q];
        if (band[q] >= 0 && last) atomicMax(&skey[band[q] - t.band_lo], run);
      }
    }
  }
  if (SELECT) {
    s1 = warp_sum64(s1);
    s2 = warp_sum64(s2);
    if (lane == 0 && (s1 | s2)) {
      atomicAdd(&md.sums[0], (unsigned long long)s1);
      atomicAdd(&md.sums[1], (unsigned long long)s2);
    }
    __syncthreads();
    for (int i = tid; i < nb_tile; i += NT)
      if (skey[i]) atomicMax(&md.keys[t.band_lo + i], skey[i]);
  }
}

// Persistent blocks over the plan's n_tiles tiles (every map of the plan in one launch): each block
// takes the next tile from the counter `next` (zeroed before the launch) until none is left.  The
// plan lists the tiles longest first, so the blocks finish together.  The index of a block's next
// tile is claimed when it starts a tile and read when it has finished it, so the atomic's round
// trip is hidden behind the tile.
template <int R, int NT, bool SELECT, bool XD, int LDS = 0, bool UNIF = false>
__global__ void __launch_bounds__(NT, NT == 1024 ? 1 : (R <= 4 ? 3 : (R == 8 ? 2 : 1)))
k_hough(const MapDev* __restrict__ maps, const TileDev* __restrict__ tiles, int n_tiles,
        int* __restrict__ next, const uint32_t* __restrict__ fft_idx,
        const uint32_t* __restrict__ bins, unsigned int* __restrict__ flag, int c_max) {
  extern __shared__ __align__(16) unsigned char smem[];
  __shared__ int s_next;
  if (threadIdx.x == 0) s_next = atomicAdd(next, 1);
  __syncthreads();
  int ti = s_next;
  while (ti < n_tiles) {
    __syncthreads();                                  // every thread has read s_next
    int claimed = 0;
    if (threadIdx.x == 0) claimed = atomicAdd(next, 1);
    const TileDev t = tiles[ti];
    if (t.nrows > 0)
      hough_tile<R, NT, SELECT, XD, LDS, UNIF>(maps, t, fft_idx, bins, flag, c_max, smem);
    if (threadIdx.x == 0) s_next = claimed;
    __syncthreads();
    ti = s_next;
  }
}

// Persistent blocks over a tile list whose length is known on the device only (the coarse-tile
// search): each block takes the next tile from a counter until the list is exhausted.  Its tiles
// are mostly narrow (a coarse tile's columns), where many warps mix interior peaks with peaks near
// an edge, so it always draws one form per warp, and tiles flagged `sub` walk only their bins'
// FFT sub-ranges (hough_tile).
template <int R, int NT, bool SELECT>
__global__ void __launch_bounds__(NT, NT == 1024 ? 1 : (R <= 4 ? 3 : (R == 8 ? 2 : 1)))
k_hough_list(const MapDev* __restrict__ maps, const TileDev* __restrict__ tiles,
             const int* __restrict__ count, int* __restrict__ next, int cap,
             const uint32_t* __restrict__ fft_idx, const uint32_t* __restrict__ bins,
             unsigned int* __restrict__ flag, int c_max, const CoarseMapDev* __restrict__ cmaps,
             const int* __restrict__ fft_unsorted, int sub_cap) {
  extern __shared__ __align__(16) unsigned char smem[];
  __shared__ int s_next;
  const int n = min(*count, cap);
  if (threadIdx.x == 0) s_next = atomicAdd(next, 1);
  __syncthreads();
  int ti = s_next;
  while (ti < n) {                                    // next tile claimed during this one
    __syncthreads();
    int claimed = 0;
    if (threadIdx.x == 0) claimed = atomicAdd(next, 1);
    const TileDev t = tiles[ti];
    if (t.nrows > 0)
      hough_tile<R, NT, SELECT, false, 0, true, true>(maps, t, fft_idx, bins, flag, c_max, smem,
                                                      cmaps, fft_unsorted, sub_cap);
    if (threadIdx.x == 0) s_next = claimed;
    __syncthreads();
    ti = s_next;
  }
}

// ---- candidate records ----------------------------------------------------------------------------

// One thread per (map, band).  Every floating-point step uses an explicitly rounded intrinsic so
// no multiply-add is contracted: the records equal a plain IEEE double evaluation.
__global__ void k_finalize(const MapDev* __restrict__ maps) {
  const MapDev& md = maps[blockIdx.y];
  const int b = blockIdx.x * blockDim.x + threadIdx.x;
  if (b >= md.n_bands) return;
  const unsigned long long s1u = md.sums[0], s2u = md.sums[1];
  const double cells = (double)md.cells;
  double mu = 0.0, sigma = 0.0;
  if (md.cells > 0) {
    mu = __ddiv_rn((double)(long long)s1u, cells);
    const double var = __dsub_rn(__ddiv_rn((double)(long long)s2u, cells), __dmul_rn(mu, mu));
    sigma = var > 0.0 ? __dsqrt_rn(var) : 0.0;
  }
  if (b == 0 && md.stats) {
    md.stats->sum = (int64_t)s1u;
    md.stats->sum_sq = (int64_t)s2u;
    md.stats->cells = md.cells;
  }
  if (!md.cands) return;
  gfh_candidate c;
  c.band = b;
  c.reserved = 0;
  const unsigned long long key = md.keys[b];
  if (key == 0ull) {
    c.row = -1; c.col = -1; c.count = -1;
    c.cr = 0.0; c.x0 = 0.0; c.k = 0.0; c.f0 = 0.0; c.fdot0 = 0.0;
  } else {
    const int count = (int)(key >> 32);
    const uint32_t lin = 0xffffffffu - (uint32_t)(key & 0xffffffffull);
    const int row = (int)(lin / (uint32_t)md.W);
    const int64_t col = (int64_t)(lin % (uint32_t)md.W);
    c.row = row;
    c.col = col;
    c.count = count;
    c.cr = sigma > 0.0 ? __ddiv_rn(__dsub_rn((double)count, mu), sigma) : 0.0;
    c.x0 = __dadd_rn(md.x0_min, __dmul_rn(__dadd_rn((double)col, 0.5), md.dx0));
    c.k = __dadd_rn(md.k_min, __dmul_rn((double)row, md.dk));
    c.f0 = md.f0c[col];
    c.fdot0 = -__dmul_rn(c.k, md.f0n[col]);
  }
  md.cands[b] = c;
}

// Selection alone on an existing map: one thread per column walks all rows.
__global__ void k_select_cols(const int32_t* __restrict__ map, const MapDev* __restrict__ mdp) {
  const MapDev& md = *mdp;
  const int64_t m = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  long long s1 = 0, s2 = 0;
  if (m < md.W) {
    const int band = md.col_band[m];
    if (band >= 0) {
      unsigned long long best = 0ull;
      for (int r = 0; r < md.K; ++r) {
        const int v = map[(int64_t)r * md.ld + m];
        s1 += v;
        s2 += (long long)v * v;
        const unsigned long long k = cand_key(v, (uint32_t)r * (uint32_t)md.W + (uint32_t)m);
        best = k > best ? k : best;
      }
      atomicMax(&md.keys[band], best);
    }
  }
  s1 = warp_sum64(s1);
  s2 = warp_sum64(s2);
  if ((threadIdx.x & 31) == 0 && (s1 | s2)) {
    atomicAdd(&md.sums[0], (unsigned long long)s1);
    atomicAdd(&md.sums[1], (unsigned long long)s2);
  }
}

// Launch (prepare = false) or set the shared-memory attribute (prepare = true).  Setting the
// attribute at plan creation keeps gfh_plan_execute to stream operations only (capturable).  The
// attribute belongs to the kernel, not to a plan, so it is set to the largest size any plan may
// request: each launch still asks only for its own size (which alone decides occupancy).
// n_tiles < 0: the persistent list form over p->d_sel_tiles with its device-side count.
// xd: the x-direction form (tiles of maps with large shifts per k row).
template <int R, int NT, bool SEL>
int launch_hough_t(gfh_plan* p, const gfh_peaks* peaks, const TileDev* tiles, int n_tiles,
                   size_t smem, bool prepare, bool xd) {
  // the shapes the autotuner picks on the paper-shaped workloads (8-row tiles of 2048 or 3072
  // columns at 512 threads, 16-row tiles of 3072 columns at 1024 threads) have the row stride
  // fixed at compile time
  // drawing form 1: one form per warp
  const bool unif = p->cfg.form == 1;
  auto fk = unif ? k_hough<R, NT, SEL, false, 0, true> : k_hough<R, NT, SEL, false>;
  if constexpr (R == 8 && NT == 512) {
    if (p->cfg.cols == 3072) fk = unif ? k_hough<R, NT, SEL, false, 3074, true> : k_hough<R, NT, SEL, false, 3074>;
    if (p->cfg.cols == 2048) fk = unif ? k_hough<R, NT, SEL, false, 2050, true> : k_hough<R, NT, SEL, false, 2050>;
  }
  if constexpr (R == 16 && NT == 1024) {
    if (p->cfg.cols == 3072) fk = unif ? k_hough<R, NT, SEL, false, 3074, true> : k_hough<R, NT, SEL, false, 3074>;
  }
  auto fn = xd ? k_hough<R, NT, SEL, true> : fk;
  auto fl = k_hough_list<R, NT, SEL>;
  if (prepare) {
    // the kernels this plan launches; each also holds a few bytes of static shared memory (the
    // tile counter)
    auto set_max = [](const void* f) -> int {
      cudaFuncAttributes fa{};
      GFH_CUDA_TRY(cudaFuncGetAttributes(&fa, f));
      GFH_CUDA_TRY(cudaFuncSetAttribute(f, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                        (int)(kMaxSmemBytes - fa.sharedSizeBytes)));
      return GFH_OK;
    };
    int rc = set_max((const void*)fk);
    if (!rc) rc = set_max((const void*)k_hough<R, NT, SEL, true>);
    if (!rc) rc = set_max((const void*)fl);
    return rc;
  }
  if (smem > kHoughSmemLimit) return GFH_ERR_SIZE;
  if (n_tiles >= 0) {
    if (n_tiles == 0) return GFH_OK;
    int per_sm = 0;
    GFH_CUDA_TRY(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, fn, NT, smem));
    const int grid = std::min(n_tiles, p->ctx->num_sms * (per_sm > 0 ? per_sm : 1));
    fn<<<grid, NT, smem, p->ctx->stream>>>(p->d_maps, tiles, n_tiles, p->d_next + (xd ? 1 : 0),
                                           peaks->fft_idx, peaks->bin, p->ctx->d_flag,
                                           p->cfg.cols);
  } else {
    int per_sm = 0;
    GFH_CUDA_TRY(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, fl, NT, smem));
    const int grid = p->ctx->num_sms * (per_sm > 0 ? per_sm : 1);
    fl<<<grid, NT, smem, p->ctx->stream>>>(p->d_maps, tiles, p->d_sel_count, p->d_sel_count + 1,
                                           p->sel_cap, peaks->fft_idx, peaks->bin, p->ctx->d_flag,
                                           p->cfg.cols, p->d_cmaps, p->d_fft_unsorted, p->sub_cap);
  }
  GFH_CUDA_TRY(cudaGetLastError());
  return GFH_OK;
}

template <int R, int NT>
int launch_hough_sel(gfh_plan* p, const gfh_peaks* peaks, const TileDev* tiles, int n_tiles,
                     size_t smem, bool prepare, bool xd) {
  return p->select ? launch_hough_t<R, NT, true>(p, peaks, tiles, n_tiles, smem, prepare, xd)
                   : launch_hough_t<R, NT, false>(p, peaks, tiles, n_tiles, smem, prepare, xd);
}

template <int R>
int launch_hough_r(gfh_plan* p, const gfh_peaks* peaks, const TileDev* tiles, int n_tiles,
                   size_t smem, bool prepare, bool xd) {
  if constexpr (R >= 16)   // 1024 threads: one block of 32 warps per SM holds a 16- or 32-row tile
    if (p->cfg.threads == 1024) return launch_hough_sel<R, 1024>(p, peaks, tiles, n_tiles, smem, prepare, xd);
  return p->cfg.threads == 256
             ? launch_hough_sel<R, 256>(p, peaks, tiles, n_tiles, smem, prepare, xd)
             : launch_hough_sel<R, 512>(p, peaks, tiles, n_tiles, smem, prepare, xd);
}

int launch_hough(gfh_plan* p, const gfh_peaks* peaks, const TileDev* tiles, int n_tiles,
                 size_t smem, bool prepare, bool xd = false) {
  return p->cfg.rows == 4    ? launch_hough_r<4>(p, peaks, tiles, n_tiles, smem, prepare, xd)
         : p->cfg.rows == 8  ? launch_hough_r<8>(p, peaks, tiles, n_tiles, smem, prepare, xd)
         : p->cfg.rows == 16 ? launch_hough_r<16>(p, peaks, tiles, n_tiles, smem, prepare, xd)
                             : launch_hough_r<32>(p, peaks, tiles, n_tiles, smem, prepare, xd);
}

// Appends to one compact list the fine tiles of each map's selected coarse tiles, or, for a map
// flagged for a full search, all tiles of the map (group nct of the map).  count[0] = list length.
// The list holds at most cap tiles (enough unless a map lists a coarse tile twice): slots are
// claimed in contiguous ranges, every claimed slot below cap is written, and an overflow sets the
// capacity flag (the list kernel reads min(count, cap) tiles).
__global__ void k_gather_tiles(const TileDev* __restrict__ fine, const int32_t* __restrict__ first,
                               const int32_t* __restrict__ coarse, const int32_t* __restrict__ full,
                               int n_sel, int nct, TileDev* __restrict__ out, int* count, int cap,
                               unsigned int* flag) {
  const int m = blockIdx.y, s = blockIdx.x;
  const bool whole = full && full[m] != 0;
  int id;
  if (whole) id = s == 0 ? nct : -1;                // one block copies the whole map
  else if (s < n_sel) id = coarse[(int64_t)m * n_sel + s];
  else return;
  if (id < 0 || id > nct || (id == nct && !whole)) return;
  const int b = first[(int64_t)m * (nct + 1) + id];
  const int e = first[(int64_t)m * (nct + 1) + id + 1];
  if (e <= b) return;
  __shared__ int base;
  if (threadIdx.x == 0) {
    base = atomicAdd(count, e - b);
    if (base + (e - b) > cap) atomicOr(flag, GFH_FLAG_CAPACITY);
  }
  __syncthreads();
  for (int q = threadIdx.x; q < e - b && base + q < cap; q += blockDim.x) out[base + q] = fine[b + q];
}

}  // namespace

size_t gfh_hough_smem_bytes(const gfh_plan* p, bool xd) {
  return (size_t)p->cfg.rows * (p->cfg.cols + 2) * 4 + (size_t)kLane * 4 * (xd ? p->cfg.rows : 1) +
         (p->select ? (size_t)p->max_tile_bands * 8 : 0);
}

int gfh_prepare_plan(gfh_plan* p) {
  const size_t smem = gfh_hough_smem_bytes(p, p->n_tiles_x > 0);
  if (smem > kHoughSmemLimit) return GFH_ERR_SIZE;
  return launch_hough(p, nullptr, nullptr, 0, smem, true);
}

// Per-execute preparation shared by the full and the coarse-tile forms: input check, per-map CSR
// over bins, zeroed candidate keys.
static int launch_prologue(gfh_plan* p, const gfh_peaks* peaks, bool coarse = false) {
  gfh_ctx* ctx = p->ctx;
  cudaStream_t st = ctx->stream;
  coarse = coarse && p->d_fft_unsorted;
  if (coarse)
    GFH_CUDA_TRY(cudaMemsetAsync(p->d_fft_unsorted, 0, sizeof(int) * p->n_list_flags, st));
  {
    dim3 grid(64, peaks->n_lists);
    k_check_sorted<<<grid, 256, 0, st>>>(peaks->bin, peaks->fft_idx, peaks->offsets, ctx->d_flag,
                                         coarse ? p->d_fft_unsorted : nullptr, p->n_list_flags);
    GFH_CUDA_TRY(cudaGetLastError());
  }
  k_csr<<<(p->csr_entries + 255) / 256, 256, 0, st>>>(p->d_maps, p->d_csr_map, p->csr_entries,
                                                      peaks->bin, peaks->offsets);
  GFH_CUDA_TRY(cudaGetLastError());
  if (coarse && p->fblk_entries > 0) {
    k_fft_blocks<<<dim3((p->fblk_entries + 255) / 256, p->n_maps), 256, 0, st>>>(
        p->d_maps, p->d_cmaps, peaks->fft_idx);
    GFH_CUDA_TRY(cudaGetLastError());
  }
  if (p->select)
    GFH_CUDA_TRY(cudaMemsetAsync(p->d_keys, 0, p->key_words * sizeof(unsigned long long), st));
  return GFH_OK;
}

static int launch_epilogue(gfh_plan* p) {
  if (p->select) {
    int maxb = 1;
    for (const gfh_grid& g : p->grids) maxb = g.n_bands > maxb ? g.n_bands : maxb;
    dim3 grid((maxb + 127) / 128, p->n_maps);
    k_finalize<<<grid, 128, 0, p->ctx->stream>>>(p->d_maps);
    GFH_CUDA_TRY(cudaGetLastError());
  }
  return GFH_OK;
}

int gfh_launch_plan(gfh_plan* p, const gfh_peaks* peaks) {
  GFH_CUDA_TRY(cudaSetDevice(p->ctx->device));
  const size_t smem = gfh_hough_smem_bytes(p, false);
  const size_t smem_x = gfh_hough_smem_bytes(p, true);
  if (smem > kHoughSmemLimit || (p->n_tiles_x > 0 && smem_x > kHoughSmemLimit)) return GFH_ERR_SIZE;
  int rc = launch_prologue(p, peaks);
  if (rc) return rc;
  GFH_CUDA_TRY(cudaMemsetAsync(p->d_next, 0, 2 * sizeof(int), p->ctx->stream));
  if (p->n_tiles > 0) {
    rc = launch_hough(p, peaks, p->d_tiles, p->n_tiles, smem, false);
    if (rc) return rc;
  }
  if (p->n_tiles_x > 0) {
    rc = launch_hough(p, peaks, p->d_tiles + p->n_tiles, p->n_tiles_x, smem_x, false, true);
    if (rc) return rc;
  }
  return launch_epilogue(p);
}

int gfh_launch_plan_tiles(gfh_plan* p, const gfh_peaks* peaks, const int32_t* d_coarse, int n_sel,
                          const int32_t* d_full) {
  GFH_CUDA_TRY(cudaSetDevice(p->ctx->device));
  // the list kernel's tile, plus the FFT sub-ranges of up to sub_cap bins
  const size_t smem = gfh_hough_smem_bytes(p, false) + (size_t)p->sub_cap * 8 + 16;
  if (smem > kHoughSmemLimit) return GFH_ERR_SIZE;
  int rc = launch_prologue(p, peaks, true);
  if (rc) return rc;
  const int nct = p->coarse_k * p->coarse_x;
  cudaStream_t st = p->ctx->stream;
  GFH_CUDA_TRY(cudaMemsetAsync(p->d_sel_count, 0, 2 * sizeof(int), st));
  const int gx = n_sel > 0 ? n_sel : 1;
  if (n_sel > 0 || d_full) {
    k_gather_tiles<<<dim3(gx, p->n_maps), 128, 0, st>>>(p->d_fine, p->d_coarse_first, d_coarse,
                                                       d_full, n_sel, nct, p->d_sel_tiles,
                                                       p->d_sel_count, p->sel_cap, p->ctx->d_flag);
    GFH_CUDA_TRY(cudaGetLastError());
    rc = launch_hough(p, peaks, p->d_sel_tiles, -1, smem, false);
    if (rc) return rc;
  }
  return launch_epilogue(p);
}

extern "C" int gfh_hough(gfh_ctx* ctx, const uint32_t* d_fft_idx, const uint32_t* d_bin,
                         int64_t n_peaks, const gfh_grid* g, int32_t* d_map,
                         gfh_candidate* d_cands, gfh_map_stats* d_stats) {
  if (!ctx || !g || !d_map || n_peaks < 0 || (n_peaks > 0 && (!d_fft_idx || !d_bin)))
    return GFH_ERR_ARG;
  gfh_grid g1 = *g;
  g1.list = 0;
  gfh_plan* p = nullptr;
  int32_t* maps[1] = {d_map};
  gfh_candidate* cands[1] = {d_cands};
  int rc = gfh_plan_create(ctx, 1, &g1, maps, d_cands ? cands : nullptr, d_stats, nullptr, &p);
  if (rc) return rc;
  k_set_offsets<<<1, 32, 0, ctx->stream>>>(p->d_offsets_single, n_peaks);
  rc = cudaGetLastError() == cudaSuccess ? GFH_OK : GFH_ERR_CUDA;
  if (!rc) {
    // An empty list still needs valid pointers for the kernels' (never executed) loads.
    gfh_peaks pk{d_fft_idx ? d_fft_idx : (const uint32_t*)p->d_offsets_single,
                 d_bin ? d_bin : (const uint32_t*)p->d_offsets_single, p->d_offsets_single, 1};
    rc = gfh_launch_plan(p, &pk);
  }
  const int rc2 = gfh_plan_destroy(p);
  return rc ? rc : rc2;
}

extern "C" int gfh_select(gfh_ctx* ctx, const int32_t* d_map, const gfh_grid* g,
                          gfh_candidate* d_cands, gfh_map_stats* d_stats) {
  if (!ctx || !d_map || !g) return GFH_ERR_ARG;
  std::vector<int32_t> band;
  std::vector<double> f0, f0n;
  int rc = gfh_host_columns(g, band, f0, f0n);
  if (rc) return rc;
  if ((double)g->n_k * (double)g->n_x0 >= 4294967295.0) return GFH_ERR_SIZE;
  int64_t ana = 0;
  for (int64_t c = 0; c < g->n_x0; ++c) ana += band[c] >= 0;
  GFH_CUDA_TRY(cudaSetDevice(ctx->device));
  const size_t nb = (size_t)g->n_bands;
  const size_t bytes = sizeof(MapDev) + 256 + (nb + 2) * 8 + band.size() * 4 + f0.size() * 16 + 1024;
  char* buf = nullptr;
  if (cudaMalloc(&buf, bytes) != cudaSuccess) return GFH_ERR_NOMEM;
  size_t off = 0;
  auto take = [&](size_t b) { size_t o = off; off = (off + b + 255) / 256 * 256; return o; };
  const size_t o_md = take(sizeof(MapDev)), o_keys = take((nb + 2) * 8),
               o_band = take(band.size() * 4), o_f0 = take(f0.size() * 8),
               o_f0n = take(f0n.size() * 8);
  MapDev md{};
  md.out = nullptr;
  md.col_band = (const int32_t*)(buf + o_band);
  md.f0c = (const double*)(buf + o_f0);
  md.f0n = (const double*)(buf + o_f0n);
  md.keys = (unsigned long long*)(buf + o_keys);
  md.sums = md.keys + nb;
  md.cands = d_cands;
  md.stats = d_stats;
  md.W = g->n_x0;
  md.ld = g->ld_x0;
  md.cells = ana * g->n_k;
  md.x0_min = g->x0_min;
  md.dx0 = g->dx0;
  md.k_min = g->k_min;
  md.dk = g->dk;
  md.K = g->n_k;
  md.n_bands = g->n_bands;
  cudaStream_t st = ctx->stream;
  cudaError_t e = cudaMemcpyAsync(buf + o_md, &md, sizeof(md), cudaMemcpyHostToDevice, st);
  if (e == cudaSuccess) e = cudaMemcpyAsync(buf + o_band, band.data(), band.size() * 4, cudaMemcpyHostToDevice, st);
  if (e == cudaSuccess) e = cudaMemcpyAsync(buf + o_f0, f0.data(), f0.size() * 8, cudaMemcpyHostToDevice, st);
  if (e == cudaSuccess) e = cudaMemcpyAsync(buf + o_f0n, f0n.data(), f0n.size() * 8, cudaMemcpyHostToDevice, st);
  if (e == cudaSuccess) e = cudaMemsetAsync(buf + o_keys, 0, (nb + 2) * 8, st);
  if (e == cudaSuccess) {
    k_select_cols<<<(unsigned)((g->n_x0 + 255) / 256), 256, 0, st>>>(d_map, (const MapDev*)(buf + o_md));
    e = cudaGetLastError();
  }
  if (e == cudaSuccess) {
    dim3 grid((unsigned)((nb + 127) / 128), 1);
    k_finalize<<<grid, 128, 0, st>>>((const MapDev*)(buf + o_md));
    e = cudaGetLastError();
  }
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);  // host vectors must outlive the copies
  cudaFree(buf);
  return e == cudaSuccess ? GFH_OK : GFH_ERR_CUDA;
}

// ---- shared-memory atomic throughput (the denominator of the accumulator's roofline) ------------
//
// Every thread adds 1 with atomicAdd to 32-bit shared words, `iters` times, cycling over four words
// of its own (so consecutive atomics of a thread do not wait on one word).  Mode 0: lane l of warp w
// uses words w * 32 + l + 1024 q (one word per bank per warp: conflict-free); mode 1: all lanes of
// a warp use the same word (same-address); mode 2: pseudo-random words of a 32 KB array.  The
// block's elapsed SM cycles go to cycles[block]; the array's sum goes to sink[block] (kept live).
namespace {

template <int MODE>
__global__ void __launch_bounds__(1024) k_smem_atomics(int iters, long long* __restrict__ cycles,
                                                       int* __restrict__ sink) {
  __shared__ int buf[8192];
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  for (int i = tid; i < 8192; i += blockDim.x) buf[i] = 0;
  __syncthreads();
  int a[4];
#pragma unroll
  for (int q = 0; q < 4; ++q) {
    if (MODE == 0) a[q] = ((warp * 32 + lane) & 1023) + 1024 * q;
    else if (MODE == 1) a[q] = (warp & 255) * 32 + 1024 * q;
    else a[q] = (int)(gfh_mix64((uint64_t)(blockIdx.x * 1024 + tid) * 4 + q) & 8191u);
  }
  const long long t0 = clock64();
  for (int i = 0; i < iters; i += 4) {
#pragma unroll
    for (int q = 0; q < 4; ++q) atomicAdd(&buf[a[q]], 1);
  }
  __syncthreads();
  const long long t1 = clock64();
  int s = 0;
  for (int i = tid; i < 8192; i += blockDim.x) s += buf[i];
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
  if (lane == 0) atomicAdd(&sink[blockIdx.x], s);
  if (tid == 0) cycles[blockIdx.x] = t1 - t0;
}

}  // namespace

extern "C" int gfh_probe_smem_atomics(gfh_ctx* ctx, int32_t mode, int32_t blocks, int32_t threads,
                                      int32_t iters, long long* d_cycles, int32_t* d_sink) {
  if (!ctx || mode < 0 || mode > 2 || blocks < 1 || threads < 32 || threads > 1024 ||
      threads % 32 || iters < 4 || iters % 4 || !d_cycles || !d_sink)
    return GFH_ERR_ARG;
  GFH_CUDA_TRY(cudaSetDevice(ctx->device));
  if (mode == 0) k_smem_atomics<0><<<blocks, threads, 0, ctx->stream>>>(iters, d_cycles, d_sink);
  if (mode == 1) k_smem_atomics<1><<<blocks, threads, 0, ctx->stream>>>(iters, d_cycles, d_sink);
  if (mode == 2) k_smem_atomics<2><<<blocks, threads, 0, ctx->stream>>>(iters, d_cycles, d_sink);
  GFH_CUDA_TRY(cudaGetLastError());
  return GFH_OK;
}

extern "C" int gfh_device_sms(gfh_ctx* ctx, int32_t* h_sms) {
  if (!ctx || !h_sms) return GFH_ERR_ARG;
  *h_sms = ctx->num_sms;
  return GFH_OK;
}
