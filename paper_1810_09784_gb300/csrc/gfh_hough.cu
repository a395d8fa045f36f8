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

// Flags peak lists whose bins are not sorted ascending.
__global__ void k_check_sorted(const uint32_t* __restrict__ bins, const int64_t* __restrict__ off,
                               unsigned int* flag) {
  const int l = blockIdx.y;
  const int64_t b = off[l], e = off[l + 1];
  for (int64_t p = b + 1 + blockIdx.x * (int64_t)blockDim.x + threadIdx.x; p < e;
       p += (int64_t)gridDim.x * blockDim.x) {
    if (bins[p] < bins[p - 1]) atomicOr(flag, GFH_FLAG_UNSORTED);
  }
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

// ---- the accumulation + prefix + select kernel ------------------------------------------------

// Shared memory: D[R][C] int32 differential tile | tot[R][32] chunk sums | skey[bands] candidates.
template <int R, int NT, bool SELECT>
__global__ void __launch_bounds__(NT, 1)
k_hough(const MapDev* __restrict__ maps, const TileDev* __restrict__ tiles,
        const uint32_t* __restrict__ fft_idx, const uint32_t* __restrict__ bins,
        unsigned int* __restrict__ flag, int c_max) {
  extern __shared__ __align__(16) unsigned char smem[];
  constexpr int NW = NT / kLane;
  const TileDev t = tiles[blockIdx.x];
  const MapDev& md = maps[t.map];
  const int C = t.ncols;
  int* D = reinterpret_cast<int*>(smem);
  int* tot = D + R * c_max;
  unsigned long long* skey = reinterpret_cast<unsigned long long*>(tot + R * kLane);
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int nb_tile = t.band_hi >= t.band_lo ? t.band_hi - t.band_lo + 1 : 0;

  for (int i = tid; i < R * C / 4; i += NT) reinterpret_cast<int4*>(D)[i] = make_int4(0, 0, 0, 0);
  if (SELECT)
    for (int i = tid; i < nb_tile; i += NT) skey[i] = 0ull;
  __syncthreads();

  // ---- accumulate: +1 / -1 at the first / one-past-last covered column of every (peak, row)
  int carry[R];
#pragma unroll
  for (int rr = 0; rr < R; ++rr) carry[rr] = 0;
  if (t.bin_a <= t.bin_b) {
    const int64_t pb = md.csr[t.bin_a - md.bin_lo];
    const int64_t pe = md.csr[t.bin_b - md.bin_lo + 1];
    const int wm1 = (int)md.W - 1;
    const int c0 = (int)t.col0, c1 = c0 + C;
    const int nrows = t.nrows;
    const int64_t* __restrict__ U = md.U;
    const int64_t* __restrict__ Bt = md.B;
    const int64_t* __restrict__ St = md.S;
    const uint32_t nfft = (uint32_t)md.n_fft;
    for (int64_t p = pb + tid; p < pe; p += NT) {
      const uint32_t f = __ldg(fft_idx + p);
      const int jl = (int)__ldg(bins + p) - md.bin_lo;
      if (f >= nfft) { atomicOr(flag, GFH_FLAG_FFT_RANGE); continue; }
      if ((unsigned)jl > (unsigned)(md.bin_hi - md.bin_lo)) {  // only if the list is unsorted
        atomicOr(flag, GFH_FLAG_UNSORTED);
        continue;
      }
      const int64_t s_i = __ldg(St + f);
      const int64_t base = __ldg(Bt + f) + (int64_t)t.row0 * s_i;
      int64_t a = __ldg(U + jl + 1) - base;       // interval start on row row0
      int64_t b1 = __ldg(U + jl) - base - 1;      // interval end - 1
#pragma unroll
      for (int rr = 0; rr < R; ++rr) {
        if (rr < nrows) {
          const int lo = max((int)(a >> GFH_FRAC_BITS), 0);
          const int hi = min((int)(b1 >> GFH_FRAC_BITS), wm1);
          if (lo <= hi && hi >= c0 && lo < c1) {
            if (lo < c0) carry[rr] += 1;
            else atomicAdd(&D[rr * C + (lo - c0)], 1);
            if (hi + 1 < c1) atomicAdd(&D[rr * C + (hi + 1 - c0)], -1);
          }
        }
        a -= s_i;
        b1 -= s_i;
      }
    }
  }
#pragma unroll
  for (int rr = 0; rr < R; ++rr) {
    const int v = warp_sum(carry[rr]);
    if (lane == 0 && v) atomicAdd(&D[rr * C], v);
  }
  __syncthreads();

  // ---- chunk sums: chunk = 128 columns (32 lanes x 4); warp w owns chunks w, w+NW, ...
  const int nch = (C + 127) / 128;
  for (int ch = warp; ch < nch; ch += NW) {
    const int col = ch * 128 + lane * 4;
    for (int rr = 0; rr < t.nrows; ++rr) {
      int s = 0;
      if (col < C) {
        const int4 v = *reinterpret_cast<const int4*>(&D[rr * C + col]);
        s = v.x + v.y + v.z + v.w;
      }
      s = warp_sum(s);
      if (lane == 0) tot[rr * kLane + ch] = s;
    }
  }
  __syncthreads();

  // ---- running sum along x0, store, candidates
  long long s1 = 0, s2 = 0;
  const uint32_t W32 = (uint32_t)md.W;
  for (int ch = warp; ch < nch; ch += NW) {
    const int col = ch * 128 + lane * 4;
    const bool in = col < C;
    int band[4] = {-1, -1, -1, -1};
    unsigned long long best[4] = {0ull, 0ull, 0ull, 0ull};
    if (SELECT && in) {
      const int4 bv = __ldg(reinterpret_cast<const int4*>(md.col_band + t.col0 + col));
      band[0] = bv.x; band[1] = bv.y; band[2] = bv.z; band[3] = bv.w;
    }
    for (int rr = 0; rr < t.nrows; ++rr) {
      int cin = (lane < ch) ? tot[rr * kLane + lane] : 0;
      cin = warp_sum(cin);
      int4 v = make_int4(0, 0, 0, 0);
      if (in) v = *reinterpret_cast<const int4*>(&D[rr * C + col]);
      v.y += v.x; v.z += v.y; v.w += v.z;
      const int incl = warp_incl_scan(v.w, lane);
      const int add = cin + incl - v.w;
      v.x += add; v.y += add; v.z += add; v.w += add;
      if (in) {
        const int64_t row = t.row0 + rr;
        __stcs(reinterpret_cast<int4*>(md.out + row * md.ld + t.col0 + col), v);
        if (SELECT) {
          const uint32_t lin0 = (uint32_t)row * W32 + (uint32_t)(t.col0 + col);
          const int vals[4] = {v.x, v.y, v.z, v.w};
#pragma unroll
          for (int q = 0; q < 4; ++q) {
            if (band[q] >= 0) {
              s1 += vals[q];
              s2 += (long long)vals[q] * vals[q];
              const unsigned long long k = cand_key(vals[q], lin0 + q);
              best[q] = k > best[q] ? k : best[q];
            }
          }
        }
      }
    }
    if (SELECT) {
      // merge equal-band neighbours among the lane's 4 columns, then one shared atomic per run
#pragma unroll
      for (int q = 0; q < 4; ++q) {
        if (band[q] < 0) continue;
        unsigned long long k = best[q];
        while (q + 1 < 4 && band[q + 1] == band[q]) { ++q; k = best[q] > k ? best[q] : k; }
        atomicMax(&skey[band[q] - t.band_lo], k);
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

template <int R, int NT, bool SEL>
int launch_hough_t(gfh_plan* p, const gfh_peaks* peaks, size_t smem) {
  auto fn = k_hough<R, NT, SEL>;
  GFH_CUDA_TRY(cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
  fn<<<p->n_tiles, NT, smem, p->ctx->stream>>>(p->d_maps, p->d_tiles, peaks->fft_idx, peaks->bin,
                                                 p->ctx->d_flag, p->cfg.cols);
  GFH_CUDA_TRY(cudaGetLastError());
  return GFH_OK;
}

template <int R, int NT>
int launch_hough_r(gfh_plan* p, const gfh_peaks* peaks, size_t smem) {
  return p->select ? launch_hough_t<R, NT, true>(p, peaks, smem)
                   : launch_hough_t<R, NT, false>(p, peaks, smem);
}

template <int R>
int launch_hough_nt(gfh_plan* p, const gfh_peaks* peaks, size_t smem) {
  return p->cfg.threads == 256 ? launch_hough_r<R, 256>(p, peaks, smem)
                               : launch_hough_r<R, 512>(p, peaks, smem);
}

}  // namespace

size_t gfh_hough_smem_bytes(const gfh_plan* p) {
  return (size_t)p->cfg.rows * p->cfg.cols * 4 + (size_t)p->cfg.rows * kLane * 4 +
         (p->select ? (size_t)p->max_tile_bands * 8 : 0);
}

int gfh_launch_plan(gfh_plan* p, const gfh_peaks* peaks) {
  gfh_ctx* ctx = p->ctx;
  GFH_CUDA_TRY(cudaSetDevice(ctx->device));
  const size_t smem = gfh_hough_smem_bytes(p);
  if (smem > 227 * 1024) return GFH_ERR_SIZE;
  cudaStream_t st = ctx->stream;
  {
    dim3 grid(64, peaks->n_lists);
    k_check_sorted<<<grid, 256, 0, st>>>(peaks->bin, peaks->offsets, ctx->d_flag);
    GFH_CUDA_TRY(cudaGetLastError());
  }
  k_csr<<<(p->csr_entries + 255) / 256, 256, 0, st>>>(p->d_maps, p->d_csr_map, p->csr_entries,
                                                      peaks->bin, peaks->offsets);
  GFH_CUDA_TRY(cudaGetLastError());
  if (p->select)
    GFH_CUDA_TRY(cudaMemsetAsync(p->d_keys, 0, p->key_words * sizeof(unsigned long long), st));
  if (p->n_tiles > 0) {
    int rc = p->cfg.rows == 8    ? launch_hough_nt<8>(p, peaks, smem)
             : p->cfg.rows == 16 ? launch_hough_nt<16>(p, peaks, smem)
                                 : launch_hough_nt<32>(p, peaks, smem);
    if (rc) return rc;
  }
  if (p->select) {
    int maxb = 1;
    for (const gfh_grid& g : p->grids) maxb = g.n_bands > maxb ? g.n_bands : maxb;
    dim3 grid((maxb + 127) / 128, p->n_maps);
    k_finalize<<<grid, 128, 0, st>>>(p->d_maps);
    GFH_CUDA_TRY(cudaGetLastError());
  }
  return GFH_OK;
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
