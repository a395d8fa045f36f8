// Candidates per "square" of a Hough map and coincidences between candidate sets (Sec. IV).
//
// Squares: the analysis columns and the k rows are each split into equal chunks; each square gives
// its highest count and a second candidate, the highest count at least min_dk rows away from the
// first (so that a second signal, or a disturbance, in the same square is not lost).  One pass over
// the stored map keeps the best cell of every (x0 chunk, row) pair; the per-square maxima then come
// from those row maxima without touching the map again.
//
// Coincidences: for every candidate of one set, the nearest candidate of another set by the Sec. IV
// distance d = sqrt(((x0_b - x0_a)/dx0)^2 + ((k_b - k_a)/dk)^2), kept when d <= radius.
#include <vector>

#include "gfh_internal.h"

namespace {

struct SqDev {
  const int32_t* map;
  int64_t ld;
  int64_t W;          // n_x0
  int64_t ca, wa;     // first analysis column and number of analysis columns
  int n_sx, n_sk, K, min_dk;
  unsigned long long* rowkey;   // [n_sx][K]
  unsigned long long* sums;     // 2
  const double* f0c;
  const double* f0n;
  double x0_min, dx0, k_min, dk;
  int64_t cells;
  gfh_candidate* out;           // [n_sx * n_sk][2]
  gfh_map_stats* stats;
};

__device__ __forceinline__ unsigned long long sq_key(int count, uint32_t lin) {
  return ((unsigned long long)(uint32_t)count << 32) | (unsigned long long)(0xffffffffu - lin);
}

__device__ __forceinline__ unsigned long long umax64(unsigned long long a, unsigned long long b) {
  return a > b ? a : b;
}

// Block (x0 chunk i, row r): the best cell of the row inside the chunk, and the row's sums.
__global__ void __launch_bounds__(256) k_sq_rows(const SqDev* __restrict__ dp) {
  const SqDev& d = *dp;
  const int i = blockIdx.x, r = blockIdx.y;
  const int64_t c0 = d.ca + (int64_t)i * d.wa / d.n_sx;
  const int64_t c1 = d.ca + (int64_t)(i + 1) * d.wa / d.n_sx;
  const int32_t* row = d.map + (int64_t)r * d.ld;
  unsigned long long best = 0ull;
  long long s1 = 0, s2 = 0;
  for (int64_t c = c0 + threadIdx.x; c < c1; c += blockDim.x) {
    const int v = __ldg(row + c);
    s1 += v;
    s2 += (long long)v * v;
    best = umax64(best, sq_key(v, (uint32_t)(r * d.W + c)));
  }
  __shared__ unsigned long long kb[8];
  __shared__ long long sb1[8], sb2[8];
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    best = umax64(best, __shfl_xor_sync(0xffffffffu, best, o));
    s1 += __shfl_xor_sync(0xffffffffu, s1, o);
    s2 += __shfl_xor_sync(0xffffffffu, s2, o);
  }
  const int w = threadIdx.x >> 5;
  if ((threadIdx.x & 31) == 0) { kb[w] = best; sb1[w] = s1; sb2[w] = s2; }
  __syncthreads();
  if (threadIdx.x == 0) {
    for (int q = 1; q < (int)(blockDim.x >> 5); ++q) {
      best = umax64(best, kb[q]);
      s1 += sb1[q];
      s2 += sb2[q];
    }
    d.rowkey[(int64_t)i * d.K + r] = best;
    if (s1 | s2) {
      atomicAdd(&d.sums[0], (unsigned long long)s1);
      atomicAdd(&d.sums[1], (unsigned long long)s2);
    }
  }
}

__device__ void sq_record(const SqDev& d, unsigned long long key, int sq, int which, double mu,
                          double sigma) {
  gfh_candidate c;
  c.band = sq;
  c.reserved = which;
  if (key == 0ull) {
    c.row = -1; c.col = -1; c.count = -1;
    c.cr = 0.0; c.x0 = 0.0; c.k = 0.0; c.f0 = 0.0; c.fdot0 = 0.0;
  } else {
    const int count = (int)(key >> 32);
    const uint32_t lin = 0xffffffffu - (uint32_t)(key & 0xffffffffull);
    const int row = (int)(lin / (uint32_t)d.W);
    const int64_t col = (int64_t)(lin % (uint32_t)d.W);
    c.row = row;
    c.col = col;
    c.count = count;
    c.cr = sigma > 0.0 ? __ddiv_rn(__dsub_rn((double)count, mu), sigma) : 0.0;
    c.x0 = __dadd_rn(d.x0_min, __dmul_rn(__dadd_rn((double)col, 0.5), d.dx0));
    c.k = __dadd_rn(d.k_min, __dmul_rn((double)row, d.dk));
    c.f0 = d.f0c[col];
    c.fdot0 = -__dmul_rn(c.k, d.f0n[col]);
  }
  d.out[2 * sq + which] = c;
}

// One thread per square: the first candidate from the row maxima, then the best row maximum at
// least min_dk rows away from it (a row maximum is the best cell of its row in the square, so the
// best far cell is the best far row maximum).
__global__ void k_sq_final(const SqDev* __restrict__ dp) {
  const SqDev& d = *dp;
  const int sq = blockIdx.x * blockDim.x + threadIdx.x;
  if (sq >= d.n_sx * d.n_sk) return;
  const int i = sq % d.n_sx, j = sq / d.n_sx;
  const int r0 = (int)((int64_t)j * d.K / d.n_sk), r1 = (int)((int64_t)(j + 1) * d.K / d.n_sk);
  const int64_t c0 = d.ca + (int64_t)i * d.wa / d.n_sx;
  const int64_t c1 = d.ca + (int64_t)(i + 1) * d.wa / d.n_sx;
  const unsigned long long s1u = d.sums[0], s2u = d.sums[1];
  double mu = 0.0, sigma = 0.0;
  if (d.cells > 0) {
    mu = __ddiv_rn((double)(long long)s1u, (double)d.cells);
    const double var = __dsub_rn(__ddiv_rn((double)(long long)s2u, (double)d.cells), __dmul_rn(mu, mu));
    sigma = var > 0.0 ? __dsqrt_rn(var) : 0.0;
  }
  if (sq == 0 && d.stats) {
    d.stats->sum = (int64_t)s1u;
    d.stats->sum_sq = (int64_t)s2u;
    d.stats->cells = d.cells;
  }
  unsigned long long k1 = 0ull, k2 = 0ull;
  if (r1 > r0 && c1 > c0) {
    for (int r = r0; r < r1; ++r) k1 = umax64(k1, d.rowkey[(int64_t)i * d.K + r]);
    const int row1 = (int)((0xffffffffu - (uint32_t)(k1 & 0xffffffffull)) / (uint32_t)d.W);
    for (int r = r0; r < r1; ++r)
      if (r - row1 >= d.min_dk || row1 - r >= d.min_dk) k2 = umax64(k2, d.rowkey[(int64_t)i * d.K + r]);
  }
  sq_record(d, k1, sq, 0, mu, sigma);
  sq_record(d, k2, sq, 1, mu, sigma);
}

// One warp per candidate of a: lane l scans the candidates l, l + 32, ... of b, then the warp keeps
// the smallest distance with ties to the lowest index.  Every distance is the same IEEE
// evaluation as a sequential scan; the square root is taken only when the squared sum improves
// (sqrt is monotone: an equal or larger squared sum cannot give a smaller distance), so the result
// equals the sequential nearest-neighbour scan exactly.
__global__ void k_coincide(const gfh_candidate* __restrict__ a, int na,
                           const gfh_candidate* __restrict__ b, int nb, double dx0, double dk,
                           double radius, int32_t* __restrict__ match, double* __restrict__ dist) {
  const int ia = (int)(((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5);
  const int lane = threadIdx.x & 31;
  if (ia >= na) return;                        // whole warps leave together
  const gfh_candidate ca = a[ia];
  double best = 0.0, best2 = 0.0;
  int bj = -1;
  if (ca.count >= 0) {
    for (int j = lane; j < nb; j += 32) {
      if (b[j].count < 0) continue;
      const double dxn = __ddiv_rn(__dsub_rn(b[j].x0, ca.x0), dx0);
      const double dkn = __ddiv_rn(__dsub_rn(b[j].k, ca.k), dk);
      const double d2 = __dadd_rn(__dmul_rn(dxn, dxn), __dmul_rn(dkn, dkn));
      if (bj < 0 || d2 < best2) {
        const double dd = __dsqrt_rn(d2);
        if (bj < 0 || dd < best) { best = dd; best2 = d2; bj = j; }
      }
    }
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    const double ob = __shfl_xor_sync(0xffffffffu, best, o);
    const int oj = __shfl_xor_sync(0xffffffffu, bj, o);
    if (oj >= 0 && (bj < 0 || ob < best || (ob == best && oj < bj))) { best = ob; bj = oj; }
  }
  if (lane == 0) {
    match[ia] = (bj >= 0 && best <= radius) ? bj : -1;
    dist[ia] = bj >= 0 ? best : -1.0;
  }
}

}  // namespace

extern "C" int gfh_select_squares(gfh_ctx* ctx, const int32_t* d_map, const gfh_grid* g,
                                  int32_t n_sx, int32_t n_sk, int32_t min_dk,
                                  gfh_candidate* d_out, gfh_map_stats* d_stats) {
  if (!ctx || !d_map || !g || !d_out || n_sx < 1 || n_sk < 1 || min_dk < 0 ||
      (int64_t)n_sx * n_sk > (1 << 24) || n_sk > g->n_k)
    return GFH_ERR_ARG;
  if (g->n_k > 65535) return GFH_ERR_SIZE;   // one grid row of blocks per k row
  std::vector<int32_t> band;
  std::vector<double> f0, f0n;
  int rc = gfh_host_columns(g, band, f0, f0n);
  if (rc) return rc;
  if ((double)g->n_k * (double)g->n_x0 >= 4294967295.0) return GFH_ERR_SIZE;
  int64_t ca = -1, cb = -1;
  for (int64_t c = 0; c < g->n_x0; ++c)
    if (band[c] >= 0) {
      if (ca < 0) ca = c;
      if (cb >= 0 && cb != c - 1) return GFH_ERR_ARG;   // analysis columns must be contiguous
      cb = c;
    }
  const int64_t wa = ca < 0 ? 0 : cb - ca + 1;
  GFH_CUDA_TRY(cudaSetDevice(ctx->device));
  size_t off = 0;
  auto take = [&](size_t b) { size_t o = off; off = (off + b + 255) / 256 * 256; return o; };
  const size_t o_d = take(sizeof(SqDev)), o_keys = take((size_t)n_sx * g->n_k * 8),
               o_sums = take(16), o_f0 = take(f0.size() * 8), o_f0n = take(f0n.size() * 8);
  rc = ensure_scratch(ctx, off);
  if (rc) return rc;
  char* buf = (char*)ctx->pm_buf;
  SqDev d{};
  d.map = d_map;
  d.ld = g->ld_x0;
  d.W = g->n_x0;
  d.ca = ca < 0 ? 0 : ca;
  d.wa = wa;
  d.n_sx = n_sx;
  d.n_sk = n_sk;
  d.K = g->n_k;
  d.min_dk = min_dk;
  d.rowkey = (unsigned long long*)(buf + o_keys);
  d.sums = (unsigned long long*)(buf + o_sums);
  d.f0c = (const double*)(buf + o_f0);
  d.f0n = (const double*)(buf + o_f0n);
  d.x0_min = g->x0_min;
  d.dx0 = g->dx0;
  d.k_min = g->k_min;
  d.dk = g->dk;
  d.cells = wa * g->n_k;
  d.out = d_out;
  d.stats = d_stats;
  cudaStream_t st = ctx->stream;
  cudaError_t e = cudaMemcpyAsync(buf + o_d, &d, sizeof(d), cudaMemcpyHostToDevice, st);
  if (e == cudaSuccess) e = cudaMemcpyAsync(buf + o_f0, f0.data(), f0.size() * 8, cudaMemcpyHostToDevice, st);
  if (e == cudaSuccess) e = cudaMemcpyAsync(buf + o_f0n, f0n.data(), f0n.size() * 8, cudaMemcpyHostToDevice, st);
  if (e == cudaSuccess) e = cudaMemsetAsync(buf + o_keys, 0, (size_t)n_sx * g->n_k * 8, st);
  if (e == cudaSuccess) e = cudaMemsetAsync(buf + o_sums, 0, 16, st);
  if (e == cudaSuccess && wa > 0) {
    k_sq_rows<<<dim3(n_sx, g->n_k), 256, 0, st>>>((const SqDev*)(buf + o_d));
    e = cudaGetLastError();
  }
  if (e == cudaSuccess) {
    const int nsq = n_sx * n_sk;
    k_sq_final<<<(nsq + 127) / 128, 128, 0, st>>>((const SqDev*)(buf + o_d));
    e = cudaGetLastError();
  }
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);  // host vectors must outlive the copies
  return e == cudaSuccess ? GFH_OK : GFH_ERR_CUDA;
}

extern "C" int gfh_coincide(gfh_ctx* ctx, const gfh_candidate* d_a, int32_t na,
                            const gfh_candidate* d_b, int32_t nb, double dx0, double dk,
                            double radius, int32_t* d_match, double* d_dist) {
  if (!ctx || na < 0 || nb < 0 || (na > 0 && (!d_a || !d_match || !d_dist)) || (nb > 0 && !d_b) ||
      !(dx0 > 0.0) || !(dk > 0.0) || !(radius >= 0.0))
    return GFH_ERR_ARG;
  if (na == 0) return GFH_OK;
  GFH_CUDA_TRY(cudaSetDevice(ctx->device));
  k_coincide<<<(unsigned)(((int64_t)na * 32 + 255) / 256), 256, 0, ctx->stream>>>(
      d_a, na, d_b, nb, dx0, dk, radius, d_match, d_dist);
  GFH_CUDA_TRY(cudaGetLastError());
  return GFH_OK;
}
