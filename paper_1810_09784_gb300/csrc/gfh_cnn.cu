// Learned tile proposer: a small convolutional network that ranks coarse (x0, k) tiles of a Hough
// map from an image of the peakmap, so that the exact Hough can run on the top tiles only.  The
// paper names machine learning as future work (Sec. VIII); the network here is a search aid, never a
// detection statistic: every candidate still comes from the exact Hough.
//
// Architecture (bf16 activations and weights, fp32 accumulation, NHWC layout):
//   input  [B][256 t][256 f][2]   log(1 + peak count) per (t, f) cell and a constant (n - 2) / 5
//   L1 3x3  2 -> 32, stride 1, ReLU       (implicit GEMMs on tcgen05, accumulators in tensor memory)
//   L2 3x3 32 -> 32, stride 2, ReLU
//   L3 3x3 32 -> 64, stride 1, ReLU
//   L4 3x3 64 -> 64, stride 2, ReLU
//   L5 3x3 64 -> 64, stride 1, ReLU       -> [B][64 t][64 f][64]
//   mean over t                           -> [B][64 f][64]
//   head: 1-D conv over f, width 3, 64 -> 64 k tiles  -> logits[b][kt * 64 + f], plus one
//   "no signal" logit: 4097 classes, softmax cross-entropy.
// The gradient of every layer is computed by hand-written kernels: weight gradients of L1-L5 and
// input gradients of L2-L5 on tcgen05 (the bias gradients summed from the same staged tiles), the
// head on CUDA cores; every reduction runs in a fixed order, so a training step is deterministic.  AdamW updates fp32
// master weights and refreshes the bf16 copies.  Activation gradients are stored masked by their
// ReLU (the gradients in the pre-activations), so the gradient kernels stage them as they are.
#include <cuda.h>
#include <cuda_bf16.h>
#include <cudaTypedefs.h>

#include <algorithm>
#include <cmath>
#include <cstring>
#include <new>

#include "gfh_internal.h"

namespace {

constexpr int kImg = 256;
constexpr size_t kSmemPerSm = 228 * 1024;   // shared memory of one SM
constexpr int kTiles = 64;
constexpr int kClasses = kTiles * kTiles + 1;

// ---- parameter layout (flat fp32 vector) --------------------------------------------------------
struct Layout {
  size_t w[5], b[5], wh, bh, bnull, total;
};
constexpr int kCin[5] = {2, 32, 32, 64, 64};
constexpr int kCout[5] = {32, 32, 64, 64, 64};
constexpr int kStride[5] = {1, 2, 1, 2, 1};

// The head's weights, biases and no-signal bias are contiguous (one gradient reduction covers them).
Layout make_layout() {
  Layout L{};
  size_t o = 0;
  for (int l = 0; l < 5; ++l) {
    L.w[l] = o; o += (size_t)kCout[l] * 9 * kCin[l];
    L.b[l] = o; o += kCout[l];
  }
  L.wh = o; o += (size_t)kTiles * 3 * 64;
  L.bh = o; o += kTiles;
  L.bnull = o; o += 1;
  L.total = o;
  return L;
}

// Channel 0 of a pixel holding `count` peaks: bf16(float(log(1 + count))), log taken in double
// (a host-built table for small counts; fp64 is slow on this part).
__device__ __forceinline__ uint32_t pixel_word(uint32_t count, float nplane,
                                               const uint16_t* __restrict__ log_tab) {
  const uint32_t a = count < (uint32_t)kLogTable
                         ? (uint32_t)__ldg(log_tab + count)
                         : (uint32_t)__bfloat16_as_ushort(__float2bfloat16_rn((float)log1p((double)count)));
  const __nv_bfloat16 b = __float2bfloat16_rn(nplane);
  return a | ((uint32_t)__bfloat16_as_ushort(b) << 16);
}

// Image of sample b: pixel (tb, fb) counts the peaks in FFTs [tb n_fft/256, (tb+1) n_fft/256) and
// bins bin_lo + [fb nb/256, (fb+1) nb/256); channel 0 = log(1 + count), channel 1 = nplane[b].
__global__ void k_synth_images(uint64_t seed, int64_t sample0, int n_fft, int bin_lo, int nb,
                               uint32_t p_noise24, const uint32_t* __restrict__ p_track24,
                               const int32_t* __restrict__ tracks, const float* __restrict__ nplane,
                               const uint16_t* __restrict__ log_tab, uint32_t* __restrict__ img) {
  const int b = blockIdx.y;
  const int pix = blockIdx.x * blockDim.x + threadIdx.x;
  if (pix >= kImg * kImg) return;
  const int tb = pix / kImg, fb = pix % kImg;
  const int i0 = (int)((int64_t)tb * n_fft / kImg), i1 = (int)((int64_t)(tb + 1) * n_fft / kImg);
  const int j0 = bin_lo + (int)((int64_t)fb * nb / kImg), j1 = bin_lo + (int)((int64_t)(fb + 1) * nb / kImg);
  const uint64_t sample = (uint64_t)(sample0 + b);
  const int32_t* tr = tracks + (int64_t)b * n_fft;
  const uint32_t pt = p_track24[b];
  uint32_t cnt = 0;
  for (int i = i0; i < i1; ++i) {
    const int tbin = tr[i];
    for (int j = j0; j < j1; ++j)
      cnt += gfh_synth_peak(seed, sample, (uint32_t)i, (uint32_t)j, p_noise24, tbin, pt);
  }
  img[(int64_t)b * kImg * kImg + pix] = pixel_word(cnt, nplane[b], log_tab);
}

// Counts peaks per pixel: list l of the peak lists into image l (one 32-bit word per pixel,
// zeroed before).  A warp takes 32 consecutive peaks; sorted lists put runs of them in one pixel,
// so lanes with the same pixel add their count in one atomic.
__global__ void k_image_count(const uint32_t* __restrict__ fft_idx, const uint32_t* __restrict__ bin,
                              const int64_t* __restrict__ offsets, int n_fft, int bin_lo, int nb,
                              uint32_t* __restrict__ img, unsigned int* flag) {
  const int l = blockIdx.y, lane = threadIdx.x & 31;
  uint32_t* im = img + (int64_t)l * kImg * kImg;
  const int64_t p1 = offsets[l + 1];
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  // the loop runs alike on all lanes of a warp (its bound is the warp's first peak)
  for (int64_t q = offsets[l] + (int64_t)blockIdx.x * blockDim.x + (threadIdx.x - lane); q < p1;
       q += stride) {
    const int64_t p = q + lane;
    int pix = -1;
    if (p < p1) {
      const uint32_t i = fft_idx[p];
      const int64_t jl = (int64_t)bin[p] - bin_lo;
      if (i >= (uint32_t)n_fft) atomicOr(flag, GFH_FLAG_FFT_RANGE);
      else if (jl >= 0 && jl < nb) {
        // pixel whose range [tb N / 256, (tb + 1) N / 256) holds i: tb = (256 (i + 1) - 1) / N
        // (32-bit: the host keeps 256 n_fft and 256 nb below 2^32)
        const int tb = (int)(((uint32_t)kImg * (i + 1u) - 1u) / (uint32_t)n_fft);
        const int fb = (int)(((uint32_t)kImg * (uint32_t)(jl + 1) - 1u) / (uint32_t)nb);
        pix = tb * kImg + fb;
      }
    }
    const unsigned same = __match_any_sync(0xffffffffu, pix);
    if (pix >= 0 && lane == __ffs(same) - 1) atomicAdd(im + pix, (uint32_t)__popc(same));
  }
}

__global__ void k_image_finish(uint32_t* __restrict__ img, const float* __restrict__ nplane,
                               const uint16_t* __restrict__ log_tab) {
  const int pix = blockIdx.x * blockDim.x + threadIdx.x;
  uint32_t* im = img + (int64_t)blockIdx.y * kImg * kImg;
  if (pix < kImg * kImg) im[pix] = pixel_word(im[pix], nplane[blockIdx.y], log_tab);
}

// Tile proposals of one map per block.  The logits give p(d, xt) (softmax over the 4096 + 1
// classes): drift class d, x0 tile xt.  Drift class d holds tracks whose drift over the
// observation, in units of K / 64 bins, lies in [d, d + 1); on x0 tile xt (f0 in [f_a, f_b)) that
// is k tiles [floor(d gb), ceil((d + 1) ga) - 1] with ga = (f_max / f_a)^n, gb = (f_max / f_b)^n,
// since one k row drifts (f0 / f_max)^n bins.  Each class spreads its probability evenly over its
// k tiles (a tile's score sums its classes' shares in increasing d).  The tiles are ranked by score
// (ties to the lower id kt * 64 + xt): a bitonic sort in shared memory of 64-bit keys, score bits
// over the complemented id; the first n tiles leave resid_n = max(0, 1 - p(null) - their score
// sum).  With tau >= 0 the list stops at the smallest n <= k with resid_n <= tau (the rest of top is
// -1), and a map whose resid_k exceeds tau is flagged for a full search; with tau < 0 all k tiles
// are kept.  1024 threads per map: the class ranges and shares are computed once per class.  For
// k <= 512 only the k largest keys are found (radix selection) and sorted.
constexpr int kProposeSelectMax = 512;   // k up to this: selection, then a sort of k keys
__global__ void __launch_bounds__(1024) k_propose(const float* __restrict__ logits,
                                                  const float* __restrict__ gain, int k, float tau,
                                                  int32_t* __restrict__ top,
                                                  float* __restrict__ resid,
                                                  int32_t* __restrict__ full) {
  constexpr int NT = 1024, NCT = kTiles * kTiles, PER = NCT / NT;
  // one 32 KB region: first the classes' shares and ranges, then the tiles' sort keys
  __shared__ __align__(16) unsigned char sbuf[NCT * 8];
  unsigned long long* key = reinterpret_cast<unsigned long long*>(sbuf);  // score bits << 32 | (0xffff - tile id)
  float* w = reinterpret_cast<float*>(sbuf);          // class (d, xt) at d * 64 + xt: share per k tile
  unsigned char* clo = sbuf + NCT * 4;                // its k tile range
  unsigned char* chi = sbuf + NCT * 5;
  __shared__ float ga[kTiles], gb[kTiles];
  __shared__ float red[NT / 32];
  __shared__ float s_bcast;
  const float* l = logits + (int64_t)blockIdx.x * kClasses;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  if (tid < kTiles) {
    ga[tid] = gain[((int64_t)blockIdx.x * kTiles + tid) * 2];
    gb[tid] = gain[((int64_t)blockIdx.x * kTiles + tid) * 2 + 1];
  }
  // softmax: max, then sum of exponentials (warp shuffles, then across the 32 warps)
  float mx = -INFINITY;
  for (int c = tid; c < kClasses; c += NT) mx = fmaxf(mx, l[c]);
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) mx = fmaxf(mx, __shfl_xor_sync(0xffffffffu, mx, o));
  if (lane == 0) red[warp] = mx;
  __syncthreads();
  if (warp == 0) {
    float v = red[lane];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v = fmaxf(v, __shfl_xor_sync(0xffffffffu, v, o));
    if (lane == 0) s_bcast = v;
  }
  __syncthreads();
  mx = s_bcast;
  float sum = 0.f;
  for (int c = tid; c < kClasses; c += NT) sum += expf(l[c] - mx);
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) sum += __shfl_xor_sync(0xffffffffu, sum, o);
  __syncthreads();                          // everyone has read s_bcast
  if (lane == 0) red[warp] = sum;
  __syncthreads();
  if (warp == 0) {
    float v = red[lane];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    if (lane == 0) s_bcast = v;
  }
  __syncthreads();
  const float lse = mx + logf(s_bcast);
  // each class: its k tile range and its share
  for (int c = tid; c < NCT; c += NT) {
    const int d = c / kTiles, xt = c % kTiles;
    const int lo = min(kTiles - 1, (int)floorf((float)d * gb[xt]));
    const int hi = min(kTiles - 1, max(lo, (int)ceilf((float)(d + 1) * ga[xt]) - 1));
    clo[c] = (unsigned char)lo;
    chi[c] = (unsigned char)hi;
    w[c] = expf(l[c] - lse) / (float)(hi - lo + 1);
  }
  __syncthreads();
  // each tile: the shares of the classes covering it, in increasing d (keys held in registers
  // until every thread has read the shares, whose storage they then take over)
  unsigned long long kreg[PER];
#pragma unroll
  for (int r = 0; r < PER; ++r) {
    const int c = tid + r * NT;
    const int kt = c / kTiles, xt = c % kTiles;
    float s = 0.f;
#pragma unroll 8
    for (int d = 0; d < kTiles; ++d) {
      const int q = d * kTiles + xt;
      if (kt >= clo[q] && kt <= chi[q]) s += w[q];
    }
    const uint32_t bits = s > 0.f ? __float_as_uint(s) : 0u;   // NaN and 0 rank last
    kreg[r] = ((unsigned long long)bits << 32) | (unsigned long long)(0xffffu - (uint32_t)c);
  }
  __syncthreads();
  if (k <= kProposeSelectMax) {
    // The k largest keys (all keys differ: each holds its tile id) without sorting all 4096: the
    // k-th largest key by an 8-bit-digit radix selection over its 48 significant bits (score bits
    // 63..32 and complemented id 15..0; bits 31..16 are 0), then the keys at or above it gathered
    // and sorted.
    unsigned int* hist = reinterpret_cast<unsigned int*>(sbuf + kProposeSelectMax * 8);
    __shared__ unsigned long long s_prefix;
    __shared__ int s_rank, s_count;
    unsigned long long prefix = 0ull, known = 0ull;    // digits fixed so far, and their bit mask
    int rank = k;                                      // rank still wanted among the matching keys
    for (int pass = 0; pass < 6; ++pass) {
      const int shift = pass < 4 ? 56 - 8 * pass : 8 - 8 * (pass - 4);   // 56 48 40 32 8 0
      for (int i = tid; i < 256; i += NT) hist[i] = 0u;
      __syncthreads();
#pragma unroll
      for (int r = 0; r < PER; ++r)
        if ((kreg[r] & known) == prefix) atomicAdd(&hist[(kreg[r] >> shift) & 255u], 1u);
      __syncthreads();
      if (warp == 0) {
        // lane l holds digits 255 - 8 l - 7 .. 255 - 8 l: counts of larger digits come first
        unsigned int c[8], tot = 0;
#pragma unroll
        for (int q = 0; q < 8; ++q) { c[q] = hist[255 - 8 * lane - q]; tot += c[q]; }
        unsigned int incl = tot;                       // inclusive scan over the lanes
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
          const unsigned int u = __shfl_up_sync(0xffffffffu, incl, o);
          if (lane >= o) incl += u;
        }
        unsigned int above = incl - tot;               // keys with a larger digit than this lane's
#pragma unroll
        for (int q = 0; q < 8; ++q) {
          if (above < (unsigned int)rank && above + c[q] >= (unsigned int)rank) {
            s_prefix = prefix | ((unsigned long long)(255 - 8 * lane - q) << shift);
            s_rank = rank - (int)above;
          }
          above += c[q];
        }
      }
      __syncthreads();
      prefix = s_prefix;
      rank = s_rank;
      known |= 255ull << shift;
    }
    // prefix is now the k-th largest key: gather the k keys >= it, pad to a power of two with 0
    // (every key is above 0) and sort them descending
    int P = 1;
    while (P < k) P <<= 1;
    if (tid == 0) s_count = 0;
    for (int i = tid; i < P; i += NT) key[i] = 0ull;
    __syncthreads();
#pragma unroll
    for (int r = 0; r < PER; ++r)
      if (kreg[r] >= prefix) key[atomicAdd(&s_count, 1)] = kreg[r];
    __syncthreads();
    for (int kk = 2; kk <= P; kk <<= 1) {
      for (int j = kk >> 1; j > 0; j >>= 1) {
        for (int i = tid; i < P; i += NT) {
          const int o = i ^ j;
          if (o > i) {
            const unsigned long long ki = key[i], ko = key[o];
            if (((i & kk) == 0) ? (ko > ki) : (ko < ki)) {
              key[i] = ko;
              key[o] = ki;
            }
          }
        }
        __syncthreads();
      }
    }
  } else {
#pragma unroll
    for (int r = 0; r < PER; ++r) key[tid + r * NT] = kreg[r];
    __syncthreads();
    // bitonic sort of all keys, descending
    for (int kk = 2; kk <= NCT; kk <<= 1) {
      for (int j = kk >> 1; j > 0; j >>= 1) {
        for (int i = tid; i < NCT; i += NT) {
          const int o = i ^ j;
          if (o > i) {
            const unsigned long long ki = key[i], ko = key[o];
            if (((i & kk) == 0) ? (ko > ki) : (ko < ki)) {
              key[i] = ko;
              key[o] = ki;
            }
          }
        }
        __syncthreads();
      }
    }
  }
  __shared__ int n_keep;
  if (tid == 0) {
    const float pnull = expf(l[kClasses - 1] - lse);
    float cum = 0.f, res = 1.f;
    int n = k;
    for (int q = 0; q < k; ++q) {
      cum += __uint_as_float((uint32_t)(key[q] >> 32));
      res = fmaxf(0.f, 1.f - pnull - cum);
      if (tau >= 0.f && res <= tau) { n = q + 1; break; }
    }
    n_keep = n;
    resid[blockIdx.x] = res;
    if (full) full[blockIdx.x] = (tau >= 0.f && res > tau) ? 1 : 0;
  }
  __syncthreads();
  for (int q = tid; q < k; q += NT)
    top[(int64_t)blockIdx.x * k + q] =
        q < n_keep ? (int32_t)(0xffffu - (uint32_t)(key[q] & 0xffffull)) : -1;
}

// Non-learned proposer: straight-line sums over channel 0 of an image.  Class (d, xt) is a track
// that starts (t = t0) in x0 tile xt, i.e. image columns 4 xt .. 4 xt + 3 when the image band is
// the analysis band, and drifts (d + 1/2) K / 64 bins over the observation; in time bin tb it
// sits off(d, tb) = round((2d + 1)(2tb + 1) K / (256 nb)) image columns left of its start column.
// score = the largest, over the four start columns c0, of sum_tb ch0[tb][c0 - off(d, tb)] (columns
// left of the image add 0).  Sums of bf16 values (multiples of 2^-8 when >= 1/2, below 2^13 in
// total) are exact in fp32.  z = (score - mean) / std over the image's 4096 scores; class logit =
// beta z; no-signal logit = LSE + det_c - det_a zmax (LSE = log sum_c exp(beta z_c), zmax the
// largest z), so that p(no signal) = 1 / (1 + exp(det_a zmax - det_c)): detection by the largest
// line sum, localisation by the line sums.  One block of 1024 threads per image, channel 0 (128 KB) and the
// offset table (64 KB) staged in shared memory; thread t owns x0 tile t % 64 and drift classes
// t / 64 + 16 j, j < 4, and sums its four start columns along each line together.
__global__ void __launch_bounds__(1024) k_line_scores(const uint32_t* __restrict__ img, int K,
                                                      int nb, float beta, float det_a, float det_c,
                                                      float* __restrict__ scores,
                                                      float* __restrict__ logits) {
  extern __shared__ __align__(16) uint16_t ch0[];    // [256][256] bf16 bits, then off[64][256]
  int* const offs = reinterpret_cast<int*>(ch0 + kImg * kImg);
  __shared__ float red[2][32];
  const uint32_t* im = img + (int64_t)blockIdx.x * kImg * kImg;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  for (int p = tid; p < kImg * kImg; p += blockDim.x) ch0[p] = (uint16_t)(im[p] & 0xffffu);
  const int64_t den = 256ll * nb;
  for (int e = tid; e < kTiles * kImg; e += blockDim.x) {
    const int d = e / kImg, tb = e % kImg;
    offs[e] = (int)(((int64_t)(2 * d + 1) * (2 * tb + 1) * K + 128ll * nb) / den);
  }
  __syncthreads();
  const int xt = tid % kTiles, dq = tid / kTiles;
  float sc[4];
  float s1 = 0.f, s2 = 0.f;
#pragma unroll 1
  for (int j = 0; j < 4; ++j) {
    const int d = dq + 16 * j;
    const int* const od = offs + d * kImg;
    float sum[4] = {0.f, 0.f, 0.f, 0.f};
    for (int tb = 0; tb < kImg; ++tb) {
      const int c = 4 * xt - od[tb];                // start column q = 0 on this row
      const uint16_t* const row = ch0 + tb * kImg;
#pragma unroll
      for (int q = 0; q < 4; ++q)
        if (c + q >= 0) sum[q] += __uint_as_float((uint32_t)row[c + q] << 16);
    }
    const float best = fmaxf(fmaxf(sum[0], sum[1]), fmaxf(sum[2], sum[3]));
    sc[j] = best;
    s1 += best;
    s2 += best * best;
  }
  // mean and deviation of the 4096 scores (fixed reduction order)
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    s1 += __shfl_xor_sync(0xffffffffu, s1, o);
    s2 += __shfl_xor_sync(0xffffffffu, s2, o);
  }
  if (lane == 0) { red[0][warp] = s1; red[1][warp] = s2; }
  __syncthreads();
  if (warp == 0) {
    float a = red[0][lane], b2 = red[1][lane];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      a += __shfl_xor_sync(0xffffffffu, a, o);
      b2 += __shfl_xor_sync(0xffffffffu, b2, o);
    }
    if (lane == 0) { red[0][0] = a; red[1][0] = b2; }
  }
  __syncthreads();
  const float mean = red[0][0] * (1.f / 4096.f);
  const float var = fmaxf(red[1][0] * (1.f / 4096.f) - mean * mean, 0.f);
  const float inv = var > 0.f ? 1.f / sqrtf(var) : 0.f;
  __syncthreads();                                   // red is reused below
  float* const lo = logits + (int64_t)blockIdx.x * kClasses;
  float zm = -INFINITY;
#pragma unroll
  for (int j = 0; j < 4; ++j) {
    const int c = (dq + 16 * j) * kTiles + xt;
    if (scores) scores[(int64_t)blockIdx.x * (kClasses - 1) + c] = sc[j];
    sc[j] = (sc[j] - mean) * inv;                    // z
    lo[c] = beta * sc[j];
    zm = fmaxf(zm, sc[j]);
  }
  // zmax, then LSE of beta z (max first for the exponentials)
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) zm = fmaxf(zm, __shfl_xor_sync(0xffffffffu, zm, o));
  if (lane == 0) red[0][warp] = zm;
  __syncthreads();
  if (warp == 0) {
    float v = red[0][lane];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v = fmaxf(v, __shfl_xor_sync(0xffffffffu, v, o));
    if (lane == 0) red[1][0] = v;
  }
  __syncthreads();
  zm = red[1][0];
  const float lm = beta * zm;                        // the largest class logit (beta >= 0)
  float e = 0.f;
#pragma unroll
  for (int j = 0; j < 4; ++j) e += expf(beta * sc[j] - lm);
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) e += __shfl_xor_sync(0xffffffffu, e, o);
  __syncthreads();
  if (lane == 0) red[0][warp] = e;
  __syncthreads();
  if (tid == 0) {
    float t = 0.f;
    for (int w = 0; w < 32; ++w) t += red[0][w];
    lo[kClasses - 1] = lm + logf(t) + det_c - det_a * zm;
  }
}

// ---- tensor-core helpers --------------------------------------------------------------------------

// Bit 0 / bit 1: whether the low / high bf16 half of w is positive (where a ReLU passes gradient).
__device__ __forceinline__ uint32_t pos_bits(uint32_t w) {
  const uint32_t lo = w & 0xffffu, hi = w >> 16;
  return (uint32_t)((lo & 0x7fffu) != 0u && !(lo & 0x8000u)) |
         ((uint32_t)((hi & 0x7fffu) != 0u && !(hi & 0x8000u)) << 1);
}

// Keeps each bf16 half of g whose bit (0: low half, 1: high half) is set in b2.
__device__ __forceinline__ uint32_t keep_by_bits(uint32_t g, uint32_t b2) {
  return g & (((b2 & 1u) ? 0xffffu : 0u) | ((b2 & 2u) ? 0xffff0000u : 0u));
}

__device__ __forceinline__ uint32_t pack_bf16(float lo, float hi) {
  const __nv_bfloat162 v = __floats2bfloat162_rn(lo, hi);
  return *reinterpret_cast<const uint32_t*>(&v);
}

// ---- tcgen05 helpers (5th-generation tensor cores, accumulator in tensor memory) --------------------
//
// Operands live in shared memory K-major without swizzle: "core matrices" of 8 rows x 16 bytes
// (8 bf16 along K); within a 16-wide K slice the two K halves are 128 bytes apart (leading byte
// offset) and consecutive 8-row groups 256 bytes apart (stride byte offset).

__device__ __forceinline__ uint32_t smem_u32(const void* p) {
  return (uint32_t)__cvta_generic_to_shared(p);
}

// Byte offset of element (row, k) of a K-major operand of `rows` rows in that layout.
__device__ __forceinline__ uint32_t cm_off(int row, int k, int rows) {
  return (uint32_t)((k >> 4) * (rows >> 3) * 256 + (row >> 3) * 256 + ((k >> 3) & 1) * 128 +
                    (row & 7) * 16 + (k & 7) * 2);
}

// Shared-memory matrix descriptor: start address, leading (K-direction) / stride (M/N-direction)
// byte offsets between core matrices, fixed version 1, no swizzle.
__device__ __forceinline__ uint64_t umma_desc(uint32_t addr, uint32_t lbo = 128u,
                                              uint32_t sbo = 256u) {
  return (uint64_t)((addr & 0x3FFFFu) >> 4) | ((uint64_t)((lbo >> 4) & 0x3FFFu) << 16) |
         ((uint64_t)((sbo >> 4) & 0x3FFFu) << 32) | (1ull << 46);
}

// Instruction descriptor of kind::f16: fp32 accumulator, bf16 A and B, both K-major, M x N.
__host__ __device__ constexpr uint32_t umma_idesc_bf16(int m, int n) {
  return (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(n >> 3) << 17) | ((uint32_t)(m >> 4) << 24);
}

__device__ __forceinline__ void umma_bf16(uint32_t tmem, uint64_t ad, uint64_t bd, uint32_t idesc,
                                          uint32_t accumulate) {
  asm volatile(
      "{\n.reg .pred p;\nsetp.ne.b32 p, %4, 0;\n"
      "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n" ::"r"(tmem),
      "l"(ad), "l"(bd), "r"(idesc), "r"(accumulate));
}

__device__ __forceinline__ void umma_commit(uint64_t* mbar) {
  asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
                   smem_u32(mbar)));
}

// Waits for the phase of parity `parity` of the mbarrier, at most `budget` cycles (default about a
// second at the maximum clock).
__device__ __forceinline__ bool mbar_wait(uint64_t* mbar, uint32_t parity,
                                          long long budget = 2000000000ll) {
  const long long t0 = clock64();
  for (;;) {
    uint32_t done;
    asm volatile(
        "{\n.reg .pred p;\nmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n"
        "selp.u32 %0, 1, 0, p;\n}\n"
        : "=r"(done)
        : "r"(smem_u32(mbar)), "r"(parity)
        : "memory");
    if (done) return true;
    if (clock64() - t0 > budget) return false;
  }
}

// Failure-path check of the bounded wait: one block waits on an mbarrier that nothing arrives at,
// gives up after `budget` cycles and raises the timeout flag, as the tensor-core kernels do.
__global__ void k_wait_unsignalled(long long budget, unsigned int* flag) {
  __shared__ __align__(8) uint64_t mbar;
  if (threadIdx.x == 0) asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(&mbar)), "r"(1));
  __syncthreads();
  if (threadIdx.x == 0 && !mbar_wait(&mbar, 0, budget)) atomicOr(flag, GFH_FLAG_TIMEOUT);
}

// 16 consecutive 32-bit accumulator columns of the warp's 32 lanes into v[0..15]; the values are
// valid after tmem_ld_wait.
__device__ __forceinline__ void tmem_ld16_issue(uint32_t taddr, uint32_t* v) {
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];\n"
      : "=r"(v[0]), "=r"(v[1]), "=r"(v[2]), "=r"(v[3]), "=r"(v[4]), "=r"(v[5]), "=r"(v[6]),
        "=r"(v[7]), "=r"(v[8]), "=r"(v[9]), "=r"(v[10]), "=r"(v[11]), "=r"(v[12]), "=r"(v[13]),
        "=r"(v[14]), "=r"(v[15])
      : "r"(taddr));
}
__device__ __forceinline__ void tmem_ld_wait() {
  asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
}

__device__ __forceinline__ void tmem_ld16(uint32_t taddr, uint32_t (&v)[16]) {
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];\n"
      : "=r"(v[0]), "=r"(v[1]), "=r"(v[2]), "=r"(v[3]), "=r"(v[4]), "=r"(v[5]), "=r"(v[6]),
        "=r"(v[7]), "=r"(v[8]), "=r"(v[9]), "=r"(v[10]), "=r"(v[11]), "=r"(v[12]), "=r"(v[13]),
        "=r"(v[14]), "=r"(v[15])
      : "r"(taddr));
  asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
}

__device__ __forceinline__ void tc_fence_before() {
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
}
__device__ __forceinline__ void tc_fence_after() {
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
}
__device__ __forceinline__ void async_proxy_fence() {
  asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}

// ---- forward layers and input gradients on tcgen05, TMA-fed and pipelined ---------------------------
// Implicit GEMM out[m][n] = relu(bias[n] + sum_k A[m][k] W[n][k]): m = output pixel (b, y, x),
// k = tap * CIN + ci (tap = 3 dy + dx), A[m][k] = in[b][y S + dy - 1][x S + dx - 1][ci] (zero outside
// the image); tcgen05.mma M = 128 output pixels x N = COUT x K = 16 (8-channel chunks as 16-byte
// rows of K-major core matrices, taps addressed through descriptor offsets into the staged input
// rows).  The first layer runs on its image padded to 8 channels (CIN = 8): a K slice is then two
// taps of one row, one input entry apart.  One output row of CW <= 128 columns per tile, with the
// roles of a block split so that copies, tensor-core work and the accumulator read-back of
// different tiles overlap:
//   warp 0      issues the tile's input copies with the tensor memory accelerator (TMA) into one of
//               NS stage buffers: one box per (8-channel chunk, parity) of 3 input rows x NP
//               entries x 16 bytes, zero-filled outside the image by the copy itself;
//   warp 1      holds the tensor memory (four accumulators of COUT columns) and issues the tile's
//               MMAs (tap by tap, K = 16 per MMA) once its stage is full and its accumulator free;
//               their completion frees the stage and marks the accumulator full;
//   warps 2-9   two groups of four that take alternate tiles: read the tile's accumulator back
//               (warp w: lanes 32 (w % 4) .., all COUT columns, one wait for all the loads) and
//               release it, add the bias and apply the ReLU (MODE 0; with `bits`, also store one
//               bit per channel where the stored value is positive) or multiply by the previous
//               layer's ReLU mask given as such bits (MODE 1, 2), and write bf16 through shared
//               memory and a tensor store.
// Stages and accumulators are handed over through mbarriers (copy bytes, MMA commits, arrivals); every
// wait is bounded and a wait that runs out raises the timeout flag and ends the block's loop.
// Input views for the copies (NHWC bf16, fully packed): S = 1: (CIN, W, H, B); S = 2: (CIN, 2, W/2,
// H, B), whose parity coordinate picks the even or odd input columns, so entry j of parity 0 is
// column 2 (x0 + j) - 1 and of parity 1 column 2 (x0 + j), as in k_conv_fwd_tc.
// MODE 2, the input gradient of a stride-2 layer, is split by output parity instead of running on
// inserted zeros: din[y][x] = sum over taps (dy, dx) with y + dy - 1 and x + dx - 1 even of
// G[(y + dy - 1) / 2][(x + dx - 1) / 2] Wf[dy][dx] (Wf the flipped, transposed weights of MODE 1).
// An even output row takes dy = 1 only (G row y / 2), an odd one dy = 0 and 2 (G rows (y - 1) / 2
// and (y + 1) / 2); likewise for columns.  A tile is one output row y and both column parities:
// output columns 2 (x0 + p) + px, p < CW, px = 0, 1, from the G rows Y = y / 2 and Y + 1 (a box of 2
// rows) and G columns x0 - 1 + j (entry j); each parity class's 1, 2, 2 or 4 taps are its only
// MMAs (a quarter of the multiply-adds of the zero-inserted form), into one accumulator per column
// parity, and the tile's 2 CW output pixels are one contiguous run of the row.
constexpr int kTmaThreads = 320, kTmaGroupWarps = 4, kTmaAcc = 4, kTmaMaxStages = 4;

__device__ __forceinline__ void mbar_init(uint64_t* bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count));
}
__device__ __forceinline__ void mbar_arrive(uint64_t* bar) {
  asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_u32(bar)) : "memory");
}
__device__ __forceinline__ void mbar_expect_tx(uint64_t* bar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)),
               "r"(bytes) : "memory");
}
__device__ __forceinline__ void tma_load_4d(uint32_t dst, const CUtensorMap* map, uint64_t* bar,
                                            int c0, int c1, int c2, int c3) {
  asm volatile(
      "cp.async.bulk.tensor.4d.shared::cluster.global.tile.mbarrier::complete_tx::bytes"
      " [%0], [%1, {%2, %3, %4, %5}], [%6];" ::"r"(dst), "l"(reinterpret_cast<uint64_t>(map)),
      "r"(c0), "r"(c1), "r"(c2), "r"(c3), "r"(smem_u32(bar)) : "memory");
}
__device__ __forceinline__ void tma_load_5d(uint32_t dst, const CUtensorMap* map, uint64_t* bar,
                                            int c0, int c1, int c2, int c3, int c4) {
  asm volatile(
      "cp.async.bulk.tensor.5d.shared::cluster.global.tile.mbarrier::complete_tx::bytes"
      " [%0], [%1, {%2, %3, %4, %5, %6}], [%7];" ::"r"(dst), "l"(reinterpret_cast<uint64_t>(map)),
      "r"(c0), "r"(c1), "r"(c2), "r"(c3), "r"(c4), "r"(smem_u32(bar)) : "memory");
}

// Tensor store of a shared-memory box to global memory (bulk group of the issuing thread).
__device__ __forceinline__ void tma_store_4d(const CUtensorMap* map, uint32_t src, int c0, int c1,
                                             int c2, int c3) {
  asm volatile(
      "cp.async.bulk.tensor.4d.global.shared::cta.bulk_group [%0, {%1, %2, %3, %4}], [%5];" ::"l"(
          reinterpret_cast<uint64_t>(map)), "r"(c0), "r"(c1), "r"(c2), "r"(c3), "r"(src)
      : "memory");
}
__device__ __forceinline__ void bulk_commit() { asm volatile("cp.async.bulk.commit_group;" ::: "memory"); }
__device__ __forceinline__ void bulk_wait_read0() {
  asm volatile("cp.async.bulk.wait_group.read 0;" ::: "memory");
}
__device__ __forceinline__ void bulk_wait0() { asm volatile("cp.async.bulk.wait_group 0;" ::: "memory"); }
__device__ __forceinline__ void group_bar(int id) {
  asm volatile("bar.sync %0, %1;" ::"r"(id), "r"(kTmaGroupWarps * 32) : "memory");
}
// Barrier of an epilogue group that also returns whether c held on any of its threads.
__device__ __forceinline__ bool group_any(int id, bool c) {
  uint32_t r;
  asm volatile(
      "{\n.reg .pred p, q;\nsetp.ne.u32 q, %1, 0;\nbar.red.or.pred p, %2, %3, q;\n"
      "selp.u32 %0, 1, 0, p;\n}\n"
      : "=r"(r)
      : "r"((uint32_t)c), "r"(id), "r"(kTmaGroupWarps * 32)
      : "memory");
  return r != 0;
}

// Bytes of one TMA box in shared memory (rows x np entries x 16 bytes, 128-byte aligned).
__host__ __device__ constexpr int tma_box_bytes(int np, int rows) {
  return (rows * np * 16 + 127) / 128 * 128;
}

// Taps of the stride-2 input gradient's parity class c = 2 py + px (see k_conv_tma): tap index
// 3 dy + dx, box row (0: G row y / 2, 1: the next) and entry offset jo; class c has 1, 2, 2, 4 taps.
__device__ __constant__ const int8_t kParityTaps[4][4][3] = {
    {{4, 0, 1}, {0, 0, 0}, {0, 0, 0}, {0, 0, 0}},
    {{3, 0, 1}, {5, 0, 2}, {0, 0, 0}, {0, 0, 0}},
    {{1, 0, 1}, {7, 1, 1}, {0, 0, 0}, {0, 0, 0}},
    {{0, 0, 1}, {2, 0, 2}, {6, 1, 1}, {8, 1, 2}}};

// The first layer (CIN == 8: the image padded to 8 channels, 51 KB of shared memory) keeps to 64
// registers so that three blocks share an SM; the others are held to one block by shared memory.
template <int CIN, int COUT, int S, int MODE>
__global__ void __launch_bounds__(kTmaThreads, CIN == 8 ? 3 : 1) k_conv_tma(const __grid_constant__ CUtensorMap tmap,
                                                             const __grid_constant__ CUtensorMap omap,
                                                             const __nv_bfloat16* __restrict__ w,
                                                             const float* __restrict__ bias,
                                                             const uint32_t* __restrict__ mbits,
                                                             uint32_t* __restrict__ bits,
                                                             __nv_bfloat16* __restrict__ out, int B,
                                                             int H, int ns, unsigned int* flag) {
  static_assert((CIN % 16 == 0 || (CIN == 8 && S == 1 && MODE == 0)) && (MODE == 0 || S == 1),
                "halo form; gradients on the G grid");
  constexpr int BW = COUT / 32;                      // mask words per pixel
  // CIN = 8: the first layer on its image padded to 8 channels (2 real); a K slice of 16 is two
  // taps (dx = 2 s, 2 s + 1) of one tap row, one entry apart, so a row takes 2 slices (the tap
  // dx = 3 has zero weights): 6 slices
  constexpr bool L1 = CIN == 8;
  constexpr int KR = 9 * CIN, SPT = CIN / 16, QC = L1 ? 1 : CIN / 8;
  constexpr int NSLW = L1 ? 6 : KR / 16;             // weight K slices
  constexpr int B_SL = COUT / 8 * 256;
  constexpr uint32_t IDESC = umma_idesc_bf16(128, COUT);
  constexpr int NPAR = MODE == 2 ? 2 : 1;          // column parities (accumulators) per tile
  constexpr int TCOLS = kTmaAcc * NPAR * COUT;
  extern __shared__ __align__(1024) unsigned char smem_tc[];
  __shared__ __align__(8) uint64_t full[kTmaMaxStages], empty[kTmaMaxStages], accf[kTmaAcc],
      acce[kTmaAcc];
  __shared__ uint32_t tslot;
  __shared__ float sbias[COUT];
  __shared__ volatile int s_fail;
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  // MODE 2: Ho = H output rows, each with two column parities of Hg = H / 2 columns
  constexpr int ROWS = MODE == 2 ? 2 : 3;
  const int Ho = H / S, Wt = MODE == 2 ? H / 2 : Ho;   // output rows, columns per tile row
  const int CW = Wt > 128 ? 128 : Wt, NCB = Wt / CW, NP = CW + 2;
  const int BOXB = tma_box_bytes(NP, ROWS), STAGE = QC * S * BOXB;
  const int n_tiles = B * Ho * NCB;
  // tile t: image b, output row y, first column x0 of the block (of G columns in MODE 2)
  auto geo = [&](int t, int& b, int& y, int& x0) {
    b = t / (Ho * NCB);
    const int r = t - b * (Ho * NCB);
    y = r / NCB;
    x0 = (r - y * NCB) * CW;
  };
  const uint32_t sb32 = smem_u32(smem_tc), sa32 = sb32 + (uint32_t)(NSLW * B_SL);
  // output staging of the two epilogue groups, after the stages and the MMA over-read pad, aligned
  // to the 1024-byte swizzle atom: 128 rows (pixels) of COUT bf16, 16-byte chunks swizzled as the
  // output tensor map's 128-byte (COUT = 64) or 64-byte (COUT = 32) mode expects
  constexpr int RB = COUT * 2;
  const uint32_t ob32 = (sa32 + (uint32_t)(ns * STAGE + 128 * 16) + 1023u) & ~1023u;
  auto fail = [&]() {
    s_fail = 1;
    atomicOr(flag, GFH_FLAG_TIMEOUT);
  };
  if (warp == 1) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(
                     smem_u32(&tslot)), "r"(TCOLS));
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
  }
  // weights, K-major rows of the output channel (MODE 1: transposed, taps flipped; L1: w holds the
  // layer's [co][tap][2] weights, placed at slice 2 dy + s, K element 8 h + ci for dx = 2 s + h)
  if (L1) {
    for (int e = tid; e < COUT * NSLW * 16; e += blockDim.x) {
      const int co = e / (NSLW * 16), k = e % (NSLW * 16);
      const int sl = k >> 4, hh = (k >> 3) & 1, ci = k & 7;
      const int dy = sl >> 1, dx = 2 * (sl & 1) + hh;
      *reinterpret_cast<__nv_bfloat16*>(smem_tc + cm_off(co, k, COUT)) =
          (dx < 3 && ci < 2) ? w[co * 18 + (3 * dy + dx) * 2 + ci] : __float2bfloat16_rn(0.f);
    }
  } else if (MODE == 0) {
    for (int e = tid; e < COUT * (KR / 8); e += blockDim.x) {
      const int co = e / (KR / 8), k = (e % (KR / 8)) * 8;
      *reinterpret_cast<int4*>(smem_tc + cm_off(co, k, COUT)) =
          __ldg(reinterpret_cast<const int4*>(w + co * KR + k));
    }
  } else {
    for (int e = tid; e < COUT * KR; e += blockDim.x) {
      const int n = e / KR, k = e - n * KR, tap = k / CIN, o = k - tap * CIN;
      *reinterpret_cast<__nv_bfloat16*>(smem_tc + cm_off(n, k, COUT)) = w[(o * 9 + 8 - tap) * COUT + n];
    }
  }
  for (int c = tid; c < COUT; c += blockDim.x) sbias[c] = MODE == 0 ? bias[c] : 0.f;
  if (L1) {
    // the zero-weight tap dx = 3 of the last row reads one entry past its box: zeros, not stale
    // bits (0 x NaN would poison the pixel), in the slack no copy writes
    for (int i = tid; i < (ns * STAGE + 128 * 16) / 16; i += blockDim.x)
      *reinterpret_cast<int4*>(smem_tc + NSLW * B_SL + i * 16) = make_int4(0, 0, 0, 0);
  }
  if (tid == 0) {
    for (int s = 0; s < ns; ++s) { mbar_init(&full[s], 1); mbar_init(&empty[s], 1); }
    for (int a = 0; a < kTmaAcc; ++a) { mbar_init(&accf[a], 1); mbar_init(&acce[a], kTmaGroupWarps); }
    s_fail = 0;
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  async_proxy_fence();
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = tslot;
  int issued = 0;                                    // stages (warp 0) or tiles (warp 1) issued

  if (warp == 0) {
    if (lane == 0) {
      asm volatile("prefetch.tensormap [%0];" ::"l"(reinterpret_cast<uint64_t>(&tmap)) : "memory");
      for (int t = blockIdx.x; t < n_tiles; t += gridDim.x) {
        const int slot = issued % ns, use = issued / ns;
        if (use > 0 && !mbar_wait(&empty[slot], (uint32_t)(use - 1) & 1u)) { fail(); break; }
        if (s_fail) break;
        int b, y, x0;
        geo(t, b, y, x0);
        mbar_expect_tx(&full[slot], (uint32_t)(QC * S * ROWS * 16 * NP));
        const uint32_t dst = sa32 + (uint32_t)(slot * STAGE);
#pragma unroll
        for (int q = 0; q < QC; ++q) {
          if constexpr (MODE == 2) {
            tma_load_4d(dst + (uint32_t)(q * BOXB), &tmap, &full[slot], 8 * q, x0 - 1, y >> 1, b);
          } else if constexpr (S == 1) {
            tma_load_4d(dst + (uint32_t)(q * BOXB), &tmap, &full[slot], 8 * q, x0 - 1, y - 1, b);
          } else {   // parity 0: odd columns 2 (x0 + j) - 1; parity 1: even columns 2 (x0 + j)
            tma_load_5d(dst + (uint32_t)(2 * q * BOXB), &tmap, &full[slot], 8 * q, 1, x0 - 1,
                        2 * y - 1, b);
            tma_load_5d(dst + (uint32_t)((2 * q + 1) * BOXB), &tmap, &full[slot], 8 * q, 0, x0,
                        2 * y - 1, b);
          }
        }
        ++issued;
      }
    }
  } else if (warp == 1) {
    if (lane == 0) {
      const uint64_t bd0 = umma_desc(sb32);
      for (int t = blockIdx.x; t < n_tiles; t += gridDim.x) {
        const int slot = issued % ns, acc = issued % kTmaAcc;
        if (issued >= kTmaAcc &&
            !mbar_wait(&acce[acc], (uint32_t)(issued / kTmaAcc - 1) & 1u)) { fail(); break; }
        if (!mbar_wait(&full[slot], (uint32_t)(issued / ns) & 1u)) { fail(); break; }
        if (s_fail) break;
        tc_fence_after();
        // descriptors: the stage's first entry plus the (chunk, parity, row, entry) offset of each
        // tap and K slice, in 16-byte units (all offsets stay inside the 14-bit address field)
        const uint64_t ad0 = umma_desc(sa32 + (uint32_t)(slot * STAGE), (uint32_t)(S * BOXB), 128u);
        const uint32_t d_tmem = tmem + (uint32_t)(acc * NPAR * COUT);
        if constexpr (L1) {
          // K halves one entry apart: the descriptor's leading byte offset is 16 bytes
          const uint64_t a1 = umma_desc(sa32 + (uint32_t)(slot * STAGE), 16u, 128u);
#pragma unroll
          for (int sl = 0; sl < 6; ++sl)
            umma_bf16(d_tmem, a1 + (uint64_t)((((sl >> 1) * NP + 2 * (sl & 1)) * 16) >> 4),
                      bd0 + (uint64_t)((sl * B_SL) >> 4), IDESC, sl > 0 ? 1u : 0u);
        } else if constexpr (MODE == 2) {
          int b, y, x0;
          geo(t, b, y, x0);
#pragma unroll
          for (int px = 0; px < 2; ++px) {
            const int cls = 2 * (y & 1) + px, nt = cls == 0 ? 1 : (cls == 3 ? 4 : 2);
#pragma unroll
            for (int k = 0; k < 4; ++k) {
              if (k < nt) {
                const int tap = kParityTaps[cls][k][0], row = kParityTaps[cls][k][1];
                const int jo = kParityTaps[cls][k][2];
#pragma unroll
                for (int sp = 0; sp < SPT; ++sp)
                  umma_bf16(d_tmem + (uint32_t)(px * COUT),
                            ad0 + (uint64_t)((2 * sp * BOXB + (row * NP + jo) * 16) >> 4),
                            bd0 + (uint64_t)(((tap * SPT + sp) * B_SL) >> 4), IDESC,
                            (k > 0 || sp > 0) ? 1u : 0u);
              }
            }
          }
        } else {
#pragma unroll
        for (int tap = 0; tap < 9; ++tap) {
          const int dy = tap / 3, dx = tap % 3;
          const int par = S == 1 ? 0 : (dx == 1 ? 1 : 0);
          const int jo = S == 1 ? dx : (dx == 2 ? 1 : 0);
#pragma unroll
          for (int sp = 0; sp < SPT; ++sp) {
            const int sl = tap * SPT + sp;
            umma_bf16(d_tmem, ad0 + (uint64_t)(((2 * sp * S + par) * BOXB + (dy * NP + jo) * 16) >> 4),
                      bd0 + (uint64_t)((sl * B_SL) >> 4), IDESC, sl > 0 ? 1u : 0u);
          }
        }
        }
        umma_commit(&empty[slot]);                   // the stage is free once these MMAs complete
        umma_commit(&accf[acc]);
        ++issued;
      }
    }
  } else {
    const int quarter = warp & 3, grp = (warp - 2) >> 2;
    const int p = quarter * 32 + lane;
    const bool leader = warp == 2 + 4 * grp && lane == 0;   // issues the group's output stores
    const uint32_t obuf = ob32 + (uint32_t)(grp * NPAR * 128 * RB);
    for (int i = grp, t = blockIdx.x + grp * gridDim.x; t < n_tiles; i += 2, t += 2 * gridDim.x) {
      const int acc = i % kTmaAcc;
      const bool got = mbar_wait(&accf[acc], (uint32_t)(i / kTmaAcc) & 1u);
      if (!got) fail();
      // the whole group leaves together (it shares barriers), on its own timeout or another's
      if (group_any(1 + grp, !got || s_fail != 0)) break;
      tc_fence_after();
      int b, y, x0;
      geo(t, b, y, x0);
      const bool valid = p < CW;
      const bool live = quarter * 32 < CW;           // warp-uniform: a row of the quarter is inside
      // the staging buffer is free once the group's previous store has read it
      if (leader) bulk_wait_read0();
      group_bar(1 + grp);
#pragma unroll
      for (int px = 0; px < NPAR; ++px) {
        // output pixel of this lane and parity: row q of the tile's staging (q = p, or 2 p + px)
        const int q = NPAR * p + px;
        const int64_t m = ((int64_t)b * Ho + y) * Ho + NPAR * x0 + q;
        const int swz = COUT == 64 ? (q & 7) : ((q >> 1) & 3);
        uint32_t v[COUT];
        if (live) {
          const uint32_t ta = tmem + ((uint32_t)(quarter * 32) << 16) +
                              (uint32_t)((acc * NPAR + px) * COUT);
#pragma unroll
          for (int c0 = 0; c0 < COUT; c0 += 16) tmem_ld16_issue(ta + (uint32_t)c0, v + c0);
          tmem_ld_wait();
        }
        if (px == NPAR - 1) {
          // the accumulator is in registers: hand it back before the output work
          tc_fence_before();
          __syncwarp();
          if (lane == 0) mbar_arrive(&acce[acc]);
        }
        if (live && valid) {
          uint32_t mw[BW > 0 ? BW : 1], pw[BW > 0 ? BW : 1];
#pragma unroll
          for (int k = 0; k < BW; ++k) {
            pw[k] = 0u;
            mw[k] = (MODE != 0 && mbits) ? __ldg(mbits + m * BW + k) : 0xffffffffu;
          }
#pragma unroll
          for (int c0 = 0; c0 < COUT; c0 += 8) {     // one 16-byte chunk: 8 channels
            uint32_t pk[4];
            if (MODE == 0) {
#pragma unroll
              for (int j = 0; j < 4; ++j) {
                pk[j] = pack_bf16(fmaxf(__uint_as_float(v[c0 + 2 * j]) + sbias[c0 + 2 * j], 0.f),
                                  fmaxf(__uint_as_float(v[c0 + 2 * j + 1]) + sbias[c0 + 2 * j + 1], 0.f));
                pw[c0 >> 5] |= pos_bits(pk[j]) << ((c0 & 31) + 2 * j);
              }
            } else {
              const uint32_t b8 = mw[c0 >> 5] >> (c0 & 31);
#pragma unroll
              for (int j = 0; j < 4; ++j)
                pk[j] = keep_by_bits(
                    pack_bf16(__uint_as_float(v[c0 + 2 * j]), __uint_as_float(v[c0 + 2 * j + 1])),
                    b8 >> (2 * j));
            }
            const uint32_t dst = obuf + (uint32_t)(q * RB + (((c0 >> 3) ^ swz) << 4));
            asm volatile("st.shared.v4.b32 [%0], {%1, %2, %3, %4};" ::"r"(dst), "r"(pk[0]),
                         "r"(pk[1]), "r"(pk[2]), "r"(pk[3]) : "memory");
          }
          if (MODE == 0 && bits) {
#pragma unroll
            for (int k = 0; k < BW; ++k) bits[m * BW + k] = pw[k];
          }
        }
      }
      async_proxy_fence();
      group_bar(1 + grp);
      if (leader) {
        tma_store_4d(&omap, obuf, 0, NPAR * x0, y, b);
        bulk_commit();
      }
    }
    if (leader) bulk_wait0();                        // the group's stores are complete
  }
  __syncthreads();
  if (s_fail) {
    // a wait ran out: let the copies and MMAs already issued land (bounded) before the shared and
    // tensor memory are given back
    if (tid == 0) {
      for (int s = 0; s < ns && s < issued; ++s) {
        const int last = issued - 1 - ((issued - 1 - s) % ns);   // last stage issued into slot s
        mbar_wait(&full[s], (uint32_t)(last / ns) & 1u);
      }
    }
    if (tid == 32 && issued > 0)
      mbar_wait(&accf[(issued - 1) % kTmaAcc], (uint32_t)((issued - 1) / kTmaAcc) & 1u);
    __syncthreads();
  }
  if (warp == 1) {
    tc_fence_after();
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(TCOLS));
  }
}

// ---- weight gradients on tcgen05, TMA-fed ----------------------------------------------------------
// dW[co][tap][ci] = sum_p G[p][co] X_tap[p][ci] with G the gradient in the layer's pre-activation
// (stored masked, NHWC [p][co]) and X_tap[p] the input pixel that output pixel p reads through the
// tap (zero outside the image).  Per tap a GEMM with M = 64 (co; rows >= COUT are padding, their
// accumulator rows never read), N = CIN (ci) and K = output pixels, both operands MN-major: a 16-byte
// row of a core matrix is 8 co (A) or 8 ci (B) of one pixel, as the NHWC tensors hold them.
// DYB = 3 (layers with CIN <= 32): block `chunk` keeps the accumulators of all nine taps in tensor
// memory over its chunk's tiles, so G is read once.  DYB = 1 (CIN = 64, whose nine taps would not
// fit): block (chunk, dy) keeps the taps (dy, 0..2) and G is read once per tap row.  A tile is
// WT_ROWS output rows x 64 columns of one image, its K-steps 16 output pixels of one row.  Warp 0
// copies each tile with the tensor memory accelerator into one of WT_STAGES stages:
//   G: one box per 8-co chunk c of WT_ROWS rows x 64 pixels  -> [c][row][64 px] x 16 bytes;
//   X: one box per 8-ci chunk c (and column parity for S = 2) of the input rows the tile's taps
//      read, x NP entries, zero-filled outside the image -> [c][par][row][NP] x 16 bytes: rows
//      (y0 + r) S + dy - 1 for DYB = 1, or all rows y0 S - 1 .. (y0 + WT_ROWS - 1) S + 1 for
//      DYB = 3 (tap row dy of output row r is row r S + dy of the box); entry j of parity 0 is
//      input column x0 S - 1 + j (S = 1), 2 (x0 + j) - 1 (S = 2), of parity 1 column 2 (x0 + j).
// Warp 1 issues the MMAs once a stage is full and frees it with their commit.  Tap dx's B operand is
// the same array started dx entries later (S = 1) or in the other parity (S = 2); for CIN = 8 the
// three taps are one MMA of N = 24 whose N-adjacent core matrices are one entry (16 bytes) apart.
// Core matrices: 8 pixels x 16 bytes, K-adjacent ones 128 bytes apart (the descriptor's leading
// byte offset), M/N-adjacent ones one chunk apart (its stride byte offset).  In the blocks whose
// tiles cover every output pixel once (all blocks for DYB = 3, the dy = 1 ones for DYB = 1),
// warps 2-3 also sum each staged G tile over its pixels
// (the bias gradient) before they release the stage with the MMA commit.  At the end the four
// warps read the accumulators to part[chunk][co][tap][ci] and the bias sums to
// bias_part[chunk][co] (k_sum_chunks adds the chunks in order).
// Pixel chunks (blocks per tap row) are a fixed count per layer, so the chunk sums run in the same
// order on every device: 384 for the first layer (narrow accumulators, several blocks per SM), 304
// for the other DYB = 3 layers (one block per SM, two waves of 152), 96 per tap row for DYB = 1.
constexpr int WT_ROWS = 2, WT_THREADS = 128, WT_STAGES = 4;
constexpr int WT_CHUNKS = 96, WT_CHUNKS1 = 384, WT_CHUNKS3 = 304;

// Tap rows per weight-gradient block and pixel chunks of a layer with CIN input channels.
constexpr int wgrad_dyb(int cin) { return cin <= 32 ? 3 : 1; }
constexpr int wgrad_chunks(int cin) {
  return cin == 8 ? WT_CHUNKS1 : (wgrad_dyb(cin) == 3 ? WT_CHUNKS3 : WT_CHUNKS);
}

// Row of an M = 64 accumulator held by tensor-memory lane `lane` (-1: no row): rows 16 q .. 16 q + 15
// sit in lanes 32 q .. 32 q + 15, the first half of each warp's quarter of the lanes.
__device__ __forceinline__ int wgrad_row_of_lane(int lane) {
  return (lane & 31) < 16 ? (lane >> 5) * 16 + (lane & 31) : -1;
}

template <int CIN, int COUT, int S, int DYB>
struct WgradTc {
  static constexpr int NP = S == 1 ? 66 : 65;                         // entries per (chunk, parity, row)
  static constexpr int XROWS = DYB == 1 ? WT_ROWS : (WT_ROWS - 1) * S + 3;   // input rows per tile
  static constexpr int GBOX = WT_ROWS * 64 * 16;                      // one G box
  static constexpr int XBOX = (XROWS * NP * 16 + 127) / 128 * 128;    // one X box (128-aligned)
  static constexpr int GB = (COUT / 8) * GBOX;
  static constexpr int XB = (CIN / 8) * S * XBOX;
  static constexpr int STAGE = (GB + XB + 127) / 128 * 128;
  // A reads 8 co chunks (64 rows): the padding chunks past G reach into X or the next stage
  static constexpr int PAD = (64 - COUT) / 8 * GBOX;
  static constexpr int SMEM = WT_STAGES * STAGE + PAD;
};

template <int CIN, int COUT, int S, int DYB>
__global__ void __launch_bounds__(WT_THREADS) k_wgrad_tma(const __grid_constant__ CUtensorMap gmap,
                                                          const __grid_constant__ CUtensorMap xmap,
                                                          float* __restrict__ part,
                                                          float* __restrict__ bias_part, int B, int H,
                                                          int chunks, unsigned int* flag) {
  using T = WgradTc<CIN, COUT, S, DYB>;
  constexpr int NP = T::NP;
  constexpr int NMMA = CIN == 8 ? 3 * CIN : CIN;
  constexpr uint32_t IDESC = (1u << 4) | (1u << 7) | (1u << 10) | (1u << 15) | (1u << 16) |
                             ((uint32_t)(NMMA >> 3) << 17) | ((uint32_t)(64 >> 4) << 24);
  constexpr int NACC = DYB * 3 * CIN;               // accumulator columns: (dy, dx, ci)
  constexpr uint32_t TCOLS = NACC <= 128 ? 128 : (NACC <= 256 ? 256 : 512);
  static_assert(NACC <= 512, "tensor memory holds the block's taps");
  extern __shared__ __align__(1024) unsigned char smem_w[];
  __shared__ __align__(8) uint64_t full[WT_STAGES], empty[WT_STAGES], done;
  __shared__ uint32_t tslot;
  __shared__ volatile int s_fail;
  // bias sums: 64 threads, TPC per 8-co chunk, 8 partial sums each
  constexpr int TPC = 64 / (COUT / 8);
  __shared__ float s_bias[64][8];
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int chunk = blockIdx.x, dy1 = blockIdx.y;  // gridDim.x == chunks; dy1: DYB = 1's tap row
  const bool bias_blk = DYB == 3 || dy1 == 1;
  const int Ho = H / S;
  const int tiles_per_img = (Ho / WT_ROWS) * (Ho / 64);
  const int n_tiles = B * tiles_per_img;
  const uint32_t s32 = smem_u32(smem_w);
  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(
                     smem_u32(&tslot)), "r"(TCOLS));
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
  }
  if (tid == 0) {
    // a stage is released by the MMA commit and, in the bias blocks, by warps 2 and 3
    for (int s = 0; s < WT_STAGES; ++s) { mbar_init(&full[s], 1); mbar_init(&empty[s], bias_blk ? 3 : 1); }
    mbar_init(&done, 1);
    s_fail = 0;
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = tslot;
  int issued = 0;

  if (warp == 0 && lane == 0) {
    asm volatile("prefetch.tensormap [%0];" ::"l"(reinterpret_cast<uint64_t>(&gmap)) : "memory");
    asm volatile("prefetch.tensormap [%0];" ::"l"(reinterpret_cast<uint64_t>(&xmap)) : "memory");
    for (int q = chunk; q < n_tiles; q += chunks) {
      const int slot = issued % WT_STAGES, use = issued / WT_STAGES;
      if (use > 0 && !mbar_wait(&empty[slot], (uint32_t)(use - 1) & 1u)) {
        s_fail = 1;
        atomicOr(flag, GFH_FLAG_TIMEOUT);
        break;
      }
      const int b = q / tiles_per_img, rem = q - b * tiles_per_img;
      const int rg = rem / (Ho / 64), cb = rem - rg * (Ho / 64);
      const int y0 = rg * WT_ROWS, x0 = cb * 64;
      const uint32_t st = s32 + (uint32_t)(slot * T::STAGE);
      mbar_expect_tx(&full[slot], (uint32_t)(T::GB + (CIN / 8) * S * T::XROWS * NP * 16));
#pragma unroll
      for (int c = 0; c < COUT / 8; ++c)
        tma_load_4d(st + (uint32_t)(c * T::GBOX), &gmap, &full[slot], 8 * c, x0, y0, b);
#pragma unroll
      for (int c = 0; c < CIN / 8; ++c) {
        const uint32_t xs = st + (uint32_t)(T::GB + c * S * T::XBOX);
        // first input row: y0 S - 1 (all tap rows), or (y0 S) + dy - 1 for one tap row, whose
        // S = 2 rows 2 (y0 + r) + dy - 1 come through the row traversal stride of 2
        const int yr = y0 * S - 1 + (DYB == 1 ? dy1 : 0);
        if constexpr (S == 1) {
          tma_load_4d(xs, &xmap, &full[slot], 8 * c, x0 - 1, yr, b);
        } else {
          tma_load_5d(xs, &xmap, &full[slot], 8 * c, 1, x0 - 1, yr, b);
          tma_load_5d(xs + (uint32_t)T::XBOX, &xmap, &full[slot], 8 * c, 0, x0, yr, b);
        }
      }
      ++issued;
    }
  } else if (warp == 1 && lane == 0) {
    for (int q = chunk; q < n_tiles; q += chunks) {
      const int slot = issued % WT_STAGES;
      if (!mbar_wait(&full[slot], (uint32_t)(issued / WT_STAGES) & 1u)) {
        s_fail = 1;
        atomicOr(flag, GFH_FLAG_TIMEOUT);
        break;
      }
      if (s_fail) break;
      tc_fence_after();
      const uint32_t st = s32 + (uint32_t)(slot * T::STAGE);
#pragma unroll
      for (int r = 0; r < WT_ROWS; ++r)
#pragma unroll
        for (int ks = 0; ks < 4; ++ks) {
          // A: [c][row][64 px]; B: [c][par][row][NP]
          const uint64_t ad =
              umma_desc(st + (uint32_t)((r * 64 + ks * 16) * 16), 128u, (uint32_t)T::GBOX);
          // every accumulator column group starts with the block's first K-step
          const uint32_t acc_on = (issued > 0 || r > 0 || ks > 0) ? 1u : 0u;
#pragma unroll
          for (int d = 0; d < DYB; ++d) {
            // box row of this output row's tap row, accumulator columns of the tap row
            const int xr = DYB == 1 ? r : r * S + d;
            const uint32_t tcol = tmem + (uint32_t)(d * 3 * CIN);
            if constexpr (CIN == 8) {
              const uint32_t b_addr = st + (uint32_t)(T::GB + (xr * NP + ks * 16) * 16);
              umma_bf16(tcol, ad, umma_desc(b_addr, 128u, 16u), IDESC, acc_on);
            } else {
#pragma unroll
              for (int dx = 0; dx < 3; ++dx) {
                const int par = S == 1 ? 0 : (dx == 1 ? 1 : 0);
                const int jo = S == 1 ? dx : (dx == 2 ? 1 : 0);
                const uint32_t b_addr =
                    st + (uint32_t)(T::GB + par * T::XBOX + (xr * NP + ks * 16 + jo) * 16);
                umma_bf16(tcol + (uint32_t)(dx * CIN), ad,
                          umma_desc(b_addr, 128u, (uint32_t)(S * T::XBOX)), IDESC, acc_on);
              }
            }
          }
        }
      umma_commit(&empty[slot]);
      ++issued;
    }
    umma_commit(&done);                              // every MMA issued above has completed
  }
  float bacc[8] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
  if (warp >= 2 && bias_blk) {
    // thread u sums chunk c = u / TPC over the pixels j, j + TPC, ... of each tile (rows, then
    // pixels, in order), j = u % TPC: consecutive threads read consecutive 16-byte rows
    const int u = tid - 64, c = u / TPC, j = u % TPC;
    int n = 0;
    for (int q = chunk; q < n_tiles; q += chunks, ++n) {
      const int slot = n % WT_STAGES;
      const bool got = mbar_wait(&full[slot], (uint32_t)(n / WT_STAGES) & 1u);
      if (!__all_sync(0xffffffffu, got)) {
        if (lane == 0) { s_fail = 1; atomicOr(flag, GFH_FLAG_TIMEOUT); }
        break;
      }
      if (__shfl_sync(0xffffffffu, s_fail, 0)) break;
      const unsigned char* g = smem_w + slot * T::STAGE + c * T::GBOX;
      for (int px = j; px < WT_ROWS * 64; px += TPC) {
        const uint4 w4 = *reinterpret_cast<const uint4*>(g + px * 16);
        const uint32_t wv[4] = {w4.x, w4.y, w4.z, w4.w};
#pragma unroll
        for (int e = 0; e < 4; ++e) {
          bacc[2 * e] += __uint_as_float(wv[e] << 16);
          bacc[2 * e + 1] += __uint_as_float(wv[e] & 0xffff0000u);
        }
      }
      __syncwarp();
      if (lane == 0) mbar_arrive(&empty[slot]);
    }
#pragma unroll
    for (int e = 0; e < 8; ++e) s_bias[u][e] = bacc[e];
  }
  __syncthreads();
  if (bias_blk && tid < COUT) {
    // co = tid: its chunk's TPC partial sums in order
    const int c = tid / 8, e = tid % 8;
    float sum = 0.f;
    for (int jj = 0; jj < TPC; ++jj) sum += s_bias[c * TPC + jj][e];
    bias_part[(int64_t)chunk * COUT + tid] = (chunk < n_tiles && !s_fail) ? sum : 0.f;
  }
  // accumulators -> part[chunk][co][tap][ci] (zeros for a block without tiles)
  bool ok = true;
  if (warp == 0) {
    const bool mine = mbar_wait(&done, 0u);
    ok = __all_sync(0xffffffffu, mine) != 0;
    if (lane == 0 && !ok) { s_fail = 1; atomicOr(flag, GFH_FLAG_TIMEOUT); }
  }
  __syncthreads();
  if (s_fail && tid == 0) {
    // let the copies already issued land (bounded) before the shared memory is given back
    for (int s = 0; s < WT_STAGES && s < issued; ++s) {
      const int last = issued - 1 - ((issued - 1 - s) % WT_STAGES);
      mbar_wait(&full[s], (uint32_t)(last / WT_STAGES) & 1u);
    }
  }
  tc_fence_after();
  const bool have = chunk < n_tiles && !s_fail;
  float* const dst = part + (int64_t)chunk * COUT * 9 * CIN;
  constexpr int JN = CIN < 16 ? CIN : 16;          // columns of one tap read per load
  for (int d = 0; d < DYB; ++d)
    for (int dx = 0; dx < 3; ++dx)
      for (int c0 = 0; c0 < CIN; c0 += 16) {
        const int tap = (DYB == 1 ? dy1 : d) * 3 + dx;
        uint32_t v[16];
        if (have)
          tmem_ld16(tmem + ((uint32_t)(warp * 32) << 16) + (uint32_t)((d * 3 + dx) * CIN + c0), v);
        const int co = wgrad_row_of_lane(warp * 32 + lane);
        if (co >= 0 && co < COUT) {
          float* o = dst + ((int64_t)co * 9 + tap) * CIN + c0;
#pragma unroll
          for (int j = 0; j < JN; ++j) o[j] = have ? __uint_as_float(v[j]) : 0.f;
        }
      }
  tc_fence_before();
  __syncthreads();
  if (warp == 0) asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(TCOLS));
}

// dst[e] += sum_{c < chunks} part[c * n + e], chunks in increasing order (deterministic).
__global__ void k_sum_chunks(const float* __restrict__ part, int chunks, int n,
                             float* __restrict__ dst) {
  const int e = blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= n) return;
  float s = 0.f;
  for (int c = 0; c < chunks; ++c) s += part[(int64_t)c * n + e];
  dst[e] += s;
}

// g[i] = dout[i] where out[i] > 0, else 0 (the gradient in a layer's pre-activation), n elements.
__global__ void k_mask_grad(const __nv_bfloat16* __restrict__ dout,
                            const __nv_bfloat16* __restrict__ out, __nv_bfloat16* __restrict__ g,
                            int64_t n) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) g[i] = __bfloat162float(out[i]) > 0.f ? dout[i] : __float2bfloat16_rn(0.f);
}

// The first layer's weight gradient runs on the tcgen05 weight-gradient kernel with the image's two
// channels zero-padded to eight (one 16-byte core-matrix row per pixel): out8[p][0..1] = img[p],
// out8[p][2..7] = 0.
__global__ void k_pad_channels(const uint32_t* __restrict__ img, int4* __restrict__ out8,
                               int64_t n_pix) {
  const int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (p < n_pix) out8[p] = make_int4((int)img[p], 0, 0, 0);
}

// dst[co][tap][ci] += sum_{c < chunks} part[c][co][tap][ci8] for ci < 2 (the padded layout has 8
// input channels), chunks in increasing order.
__global__ void k_sum_chunks_l1(const float* __restrict__ part, int chunks, float* __restrict__ dst) {
  const int e = blockIdx.x * blockDim.x + threadIdx.x;   // (co, tap, ci) of 32 x 9 x 2
  if (e >= 576) return;
  const int ci = e & 1, ct = e >> 1;
  float s = 0.f;
  for (int c = 0; c < chunks; ++c) s += part[(int64_t)c * 32 * 9 * 8 + ct * 8 + ci];
  dst[e] += s;
}

// ---- mean over t, head, loss --------------------------------------------------------------------
// pooled[b][f][c] = mean_t a5[b][t][f][c]
__global__ void k_pool(const __nv_bfloat16* __restrict__ a5, float* __restrict__ pooled, int B) {
  const int e = blockIdx.x * blockDim.x + threadIdx.x;   // (b, f, c)
  if (e >= B * 64 * 64) return;
  const int b = e / 4096, fc = e % 4096;
  float s = 0.f;
  for (int tt = 0; tt < 64; ++tt) s += __bfloat162float(a5[((int64_t)b * 64 + tt) * 4096 + fc]);
  pooled[e] = s * (1.0f / 64.0f);
}

// logits[b][kt * 64 + f] = bh[kt] + sum_{d, c} wh[kt][d][c] pooled[b][f + d - 1][c]; logits[b][4096]
// = bnull.  Block (q, b): image b, k tiles kt = 16 q .. 16 q + 15, their weights and the image's
// pooled rows (zero-padded rows -1 and 64) in shared memory; a thread owns one kt and 4
// consecutive f, so each weight is read once for 4 products and each pooled value once per (c, row)
// for up to 3 taps.  Every logit sums its terms in the same order (c ascending, taps d = 0, 1, 2).
constexpr int kHeadKtPerBlock = 16;
__global__ void __launch_bounds__(256) k_head_fwd(const float* __restrict__ pooled,
                                                  const float* __restrict__ wh,
                                                  const float* __restrict__ bh,
                                                  const float* __restrict__ bnull,
                                                  float* __restrict__ logits) {
  constexpr int LDP = 65;                  // padded row: rows differing in f fall in other banks
  __shared__ float pp[66 * LDP];
  __shared__ float ws[kHeadKtPerBlock * 192];
  const int b = blockIdx.y, kt0 = blockIdx.x * kHeadKtPerBlock;
  for (int e = threadIdx.x; e < 66 * 64; e += blockDim.x) {
    const int row = e / 64, c = e % 64;
    const int f = row - 1;
    pp[row * LDP + c] = (f >= 0 && f < 64) ? pooled[((int64_t)b * 64 + f) * 64 + c] : 0.f;
  }
  for (int e = threadIdx.x; e < kHeadKtPerBlock * 192; e += blockDim.x) ws[e] = wh[kt0 * 192 + e];
  __syncthreads();
  const int kl = threadIdx.x >> 4, f0 = (threadIdx.x & 15) * 4, kt = kt0 + kl;
  float acc[4];
  const float bias = bh[kt];
#pragma unroll
  for (int j = 0; j < 4; ++j) acc[j] = bias;
  const float* w = ws + kl * 192;
#pragma unroll 4
  for (int c = 0; c < 64; ++c) {
    const float w0 = w[c], w1 = w[64 + c], w2 = w[128 + c];
    float v[6];
#pragma unroll
    for (int j = 0; j < 6; ++j) v[j] = pp[(f0 + j) * LDP + c];   // rows f0 .. f0 + 5 = f - 1 ..
#pragma unroll
    for (int j = 0; j < 4; ++j) acc[j] += w0 * v[j] + w1 * v[j + 1] + w2 * v[j + 2];
  }
  float* o = logits + (int64_t)b * kClasses + kt * 64 + f0;
#pragma unroll
  for (int j = 0; j < 4; ++j) o[j] = acc[j];
  if (blockIdx.x == 0 && threadIdx.x == 0) logits[(int64_t)b * kClasses + kClasses - 1] = bnull[0];
}

// Softmax cross-entropy per sample (one block of 256 threads per sample): loss[b], and dlogits =
// (softmax - onehot) / B.
__global__ void k_softmax_ce(const float* __restrict__ logits, const int32_t* __restrict__ labels,
                             float* __restrict__ dlogits, float* __restrict__ loss, int B) {
  const int b = blockIdx.x;
  const float* l = logits + (int64_t)b * kClasses;
  __shared__ float red[256];
  float mx = -INFINITY;
  for (int c = threadIdx.x; c < kClasses; c += blockDim.x) mx = fmaxf(mx, l[c]);
  red[threadIdx.x] = mx;
  __syncthreads();
  for (int s = 128; s > 0; s >>= 1) {
    if (threadIdx.x < s) red[threadIdx.x] = fmaxf(red[threadIdx.x], red[threadIdx.x + s]);
    __syncthreads();
  }
  mx = red[0];
  __syncthreads();
  float sum = 0.f;
  for (int c = threadIdx.x; c < kClasses; c += blockDim.x) sum += expf(l[c] - mx);
  red[threadIdx.x] = sum;
  __syncthreads();
  for (int s = 128; s > 0; s >>= 1) {
    if (threadIdx.x < s) red[threadIdx.x] += red[threadIdx.x + s];
    __syncthreads();
  }
  const float lse = mx + logf(red[0]);
  const int y = labels[b];
  if (threadIdx.x == 0) loss[b] = lse - l[y];
  if (dlogits)
    for (int c = threadIdx.x; c < kClasses; c += blockDim.x)
      dlogits[(int64_t)b * kClasses + c] = (expf(l[c] - lse) - (c == y ? 1.f : 0.f)) / (float)B;
}

// Head weight/bias gradients: one thread per (kt, d, c) weight, plus bias and null bias, summing
// the images of chunk blockIdx.y (kHeadImgs images) into part[chunk][weight] (k_sum_chunks adds the
// chunks in order).
constexpr int kHeadImgs = 16, kHeadParams = 64 * 3 * 64 + 65;
__global__ void k_head_wgrad(const float* __restrict__ dlogits, const float* __restrict__ pooled,
                             float* __restrict__ part, int B) {
  const int e = blockIdx.x * blockDim.x + threadIdx.x;
  const int b0 = blockIdx.y * kHeadImgs, b1 = min(B, b0 + kHeadImgs);
  float s = 0.f;
  if (e < 64 * 3 * 64) {
    const int kt = e / 192, d = (e / 64) % 3, c = e % 64;
    for (int b = b0; b < b1; ++b)
      for (int f = 0; f < 64; ++f) {
        const int ff = f + d - 1;
        if (ff < 0 || ff >= 64) continue;
        s += dlogits[(int64_t)b * kClasses + kt * 64 + f] * pooled[((int64_t)b * 64 + ff) * 64 + c];
      }
  } else if (e < 64 * 3 * 64 + 64) {
    const int kt = e - 64 * 3 * 64;
    for (int b = b0; b < b1; ++b)
      for (int f = 0; f < 64; ++f) s += dlogits[(int64_t)b * kClasses + kt * 64 + f];
  } else if (e == 64 * 3 * 64 + 64) {
    for (int b = b0; b < b1; ++b) s += dlogits[(int64_t)b * kClasses + kClasses - 1];
  } else {
    return;
  }
  part[(int64_t)blockIdx.y * kHeadParams + e] = s;
}

// d a5[b][t][f][c] = (1/64) sum_{kt, d} dlogits[b][kt * 64 + f - d + 1] wh[kt][d][c]  (same for all t),
// stored masked by a5 > 0: the gradient in layer 5's pre-activation
__global__ void k_head_dgrad(const float* __restrict__ dlogits, const float* __restrict__ wh,
                             const __nv_bfloat16* __restrict__ a5, __nv_bfloat16* __restrict__ da5,
                             int B) {
  const int e = blockIdx.x * blockDim.x + threadIdx.x;   // (b, f, c)
  if (e >= B * 4096) return;
  const int b = e / 4096, f = (e / 64) % 64, c = e % 64;
  float s = 0.f;
  for (int kt = 0; kt < 64; ++kt)
    for (int d = 0; d < 3; ++d) {
      const int fo = f - d + 1;
      if (fo < 0 || fo >= 64) continue;
      s += dlogits[(int64_t)b * kClasses + kt * 64 + fo] * wh[(kt * 3 + d) * 64 + c];
    }
  const __nv_bfloat16 v = __float2bfloat16_rn(s * (1.0f / 64.0f));
  const __nv_bfloat16 zero = __float2bfloat16_rn(0.f);
  for (int tt = 0; tt < 64; ++tt) {
    const int64_t i = ((int64_t)b * 64 + tt) * 4096 + f * 64 + c;
    da5[i] = __bfloat162float(a5[i]) > 0.f ? v : zero;
  }
}

// AdamW on the fp32 master weights; refreshes the bf16 copies of L2-L5 (index map in bf16_of).
__global__ void k_adamw(float* __restrict__ w, const float* __restrict__ gw, float* __restrict__ m,
                        float* __restrict__ v, int64_t n, float lr, float b1, float b2, float eps,
                        float wd, float c1, float c2) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const float gi = gw[i];
  const float mi = b1 * m[i] + (1.f - b1) * gi;
  const float vi = b2 * v[i] + (1.f - b2) * gi * gi;
  m[i] = mi;
  v[i] = vi;
  w[i] -= lr * ((mi / c1) / (sqrtf(vi / c2) + eps) + wd * w[i]);
}

__global__ void k_to_bf16(const float* __restrict__ a, __nv_bfloat16* __restrict__ b, int64_t n) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) b[i] = __float2bfloat16_rn(a[i]);
}

// ---- launch helpers -------------------------------------------------------------------------------

// cuTensorMapEncodeTiled from the driver, looked up once through the runtime.
PFN_cuTensorMapEncodeTiled_v12000 tensor_map_encoder() {
  static PFN_cuTensorMapEncodeTiled_v12000 fn = [] {
    void* p = nullptr;
    cudaDriverEntryPointQueryResult q{};
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) !=
            cudaSuccess || q != cudaDriverEntryPointSuccess)
      p = nullptr;
    return reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(p);
  }();
  return fn;
}

// Launch of k_conv_tma (see there): the input view's tensor map, the stage count that fits in shared
// memory next to the weights (4, 3 or 2), persistent blocks.
template <int CIN, int COUT, int S, int MODE>
int conv_tma(const __nv_bfloat16* in, const __nv_bfloat16* w, const float* bias,
             const uint32_t* mbits, uint32_t* bits, __nv_bfloat16* out, int B, int H, int sms,
             cudaStream_t st, unsigned int* flag) {
  // MODE 2: G is H/2 x H/2; a tile covers CW of its columns, both output column parities
  constexpr int ROWS = MODE == 2 ? 2 : 3;
  const int Ho = H / S, Wt = MODE == 2 ? H / 2 : Ho;
  const int CW = Wt > 128 ? 128 : Wt, NP = CW + 2;
  if (Wt < 1 || Ho * S != H || (MODE == 2 && H % 2) || Wt % CW) return GFH_ERR_ARG;
  const PFN_cuTensorMapEncodeTiled_v12000 encode = tensor_map_encoder();
  if (!encode) return GFH_ERR_CUDA;
  alignas(64) CUtensorMap map;
  const cuuint64_t e = 2;                            // bf16 bytes
  CUresult r;
  if (MODE == 2) {
    const cuuint64_t hg = (cuuint64_t)H / 2;
    const cuuint64_t dims[4] = {(cuuint64_t)CIN, hg, hg, (cuuint64_t)B};
    const cuuint64_t strides[3] = {CIN * e, hg * CIN * e, hg * hg * CIN * e};
    const cuuint32_t box[4] = {8, (cuuint32_t)NP, 2, 1}, es[4] = {1, 1, 1, 1};
    r = encode(&map, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 4, (void*)in, dims, strides, box, es,
               CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE,
               CU_TENSOR_MAP_L2_PROMOTION_L2_128B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  } else if (S == 1) {
    const cuuint64_t dims[4] = {(cuuint64_t)CIN, (cuuint64_t)H, (cuuint64_t)H, (cuuint64_t)B};
    const cuuint64_t strides[3] = {CIN * e, (cuuint64_t)H * CIN * e, (cuuint64_t)H * H * CIN * e};
    const cuuint32_t box[4] = {8, (cuuint32_t)NP, 3, 1}, es[4] = {1, 1, 1, 1};
    r = encode(&map, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 4, (void*)in, dims, strides, box, es,
               CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE,
               CU_TENSOR_MAP_L2_PROMOTION_L2_128B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  } else {
    const cuuint64_t dims[5] = {(cuuint64_t)CIN, 2, (cuuint64_t)H / 2, (cuuint64_t)H, (cuuint64_t)B};
    const cuuint64_t strides[4] = {CIN * e, 2 * CIN * e, (cuuint64_t)H * CIN * e,
                                   (cuuint64_t)H * H * CIN * e};
    const cuuint32_t box[5] = {8, 1, (cuuint32_t)NP, 3, 1}, es[5] = {1, 1, 1, 1, 1};
    r = encode(&map, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 5, (void*)in, dims, strides, box, es,
               CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE,
               CU_TENSOR_MAP_L2_PROMOTION_L2_128B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  }
  if (r != CUDA_SUCCESS) return GFH_ERR_CUDA;
  // output view for the tensor stores: NHWC (COUT, Ho, Ho, B), boxes of one row's CW pixels (mode
  // 2: 2 CW, both column parities of the tile)
  alignas(64) CUtensorMap omap;
  const CUtensorMapSwizzle oswz = COUT == 64 ? CU_TENSOR_MAP_SWIZZLE_128B : CU_TENSOR_MAP_SWIZZLE_64B;
  static_assert(COUT == 32 || COUT == 64, "output rows of 64 or 128 bytes");
  constexpr int NPAR = MODE == 2 ? 2 : 1;
  {
    const cuuint64_t dims[4] = {(cuuint64_t)COUT, (cuuint64_t)Ho, (cuuint64_t)Ho, (cuuint64_t)B};
    const cuuint64_t strides[3] = {COUT * e, (cuuint64_t)Ho * COUT * e, (cuuint64_t)Ho * Ho * COUT * e};
    const cuuint32_t box[4] = {(cuuint32_t)COUT, (cuuint32_t)(NPAR * CW), 1, 1}, es[4] = {1, 1, 1, 1};
    r = encode(&omap, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 4, (void*)out, dims, strides, box, es,
               CU_TENSOR_MAP_INTERLEAVE_NONE, oswz, CU_TENSOR_MAP_L2_PROMOTION_NONE,
               CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  }
  if (r != CUDA_SUCCESS) return GFH_ERR_CUDA;
  auto fn = k_conv_tma<CIN, COUT, S, MODE>;
  cudaFuncAttributes fa{};
  GFH_CUDA_TRY(cudaFuncGetAttributes(&fa, fn));
  // weights, stages, the over-read of the dropped MMA rows past the last stage, then (aligned to
  // 1024 bytes) the two epilogue groups' output staging of 128 rows x COUT bf16
  const size_t w_bytes = (size_t)(CIN == 8 ? 6 : 9 * CIN / 16) * (COUT / 8 * 256);
  const size_t stage = (size_t)(CIN / 8) * S * tma_box_bytes(NP, ROWS);
  const size_t o_bytes = 2 * NPAR * 128 * COUT * 2 + 1024;
  const size_t room = kMaxSmemBytes - fa.sharedSizeBytes - 1024;
  int ns = kTmaMaxStages;
  while (ns >= 2 && w_bytes + ns * stage + 128 * 16 + o_bytes > room) --ns;
  if (ns < 2) return GFH_ERR_SIZE;
  const size_t smem = w_bytes + ns * stage + 128 * 16 + o_bytes;
  GFH_CUDA_TRY(cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
  GFH_CUDA_TRY(cudaFuncSetAttribute(fn, cudaFuncAttributePreferredSharedMemoryCarveout, 100));
  const int regs = std::max(1, (fa.numRegs + 7) / 8 * 8);
  const int per_sm = std::max(1, std::min({(int)(kSmemPerSm / (smem + fa.sharedSizeBytes + 1024)),
                                           65536 / (regs * kTmaThreads), 2048 / kTmaThreads,
                                           512 / (kTmaAcc * NPAR * COUT)}));
  const int64_t tiles = (int64_t)B * Ho * (Wt / CW);
  const int grid = (int)std::min<int64_t>(tiles, (int64_t)sms * per_sm);
  fn<<<grid, kTmaThreads, smem, st>>>(map, omap, w, bias, mbits, bits, out, B, H, ns, flag);
  GFH_CUDA_TRY(cudaGetLastError());
  return GFH_OK;
}

// One 3x3 layer: forward (MODE 0) or input gradient (MODE 1: stride-1 layer, MODE 2: stride-2
// layer; `in` the gradient in the layer's pre-activation, `w` the layer's weights).  bits (MODE 0,
// nullable): one bit per output channel, set where the stored value is positive, COUT / 32 words
// per pixel.  mbits (MODE 1, 2, nullable): such bits of the previous layer's output, the ReLU mask
// the stored gradient is multiplied by.
template <int CIN, int COUT, int S, int MODE = 0>
int conv_fwd(const __nv_bfloat16* in, const __nv_bfloat16* w, const float* bias,
             const uint32_t* mbits, uint32_t* bits, __nv_bfloat16* out, int B, int H, int sms,
             cudaStream_t st, unsigned int* flag) {
  static_assert(CIN % 16 == 0 || CIN == 8, "16-byte channel chunks (the first layer padded to 8)");
  return conv_tma<CIN, COUT, S, MODE>(in, w, bias, mbits, bits, out, B, H, sms, st, flag);
}

// The first layer's forward: the image [B][H][H][2] padded to 8 channels into img8, then the
// TMA-fed convolution on it (w: the layer's [32][3][3][2] weights).
int conv1_fwd(const __nv_bfloat16* img, __nv_bfloat16* img8, const __nv_bfloat16* w,
              const float* bias, uint32_t* bits, __nv_bfloat16* out, int B, int H, int sms,
              cudaStream_t st, unsigned int* flag) {
  const int64_t P1 = (int64_t)B * H * H;
  k_pad_channels<<<(unsigned)((P1 + 255) / 256), 256, 0, st>>>((const uint32_t*)img, (int4*)img8, P1);
  GFH_CUDA_TRY(cudaGetLastError());
  return conv_fwd<8, 32, 1>(img8, w, bias, nullptr, bits, out, B, H, sms, st, flag);
}

// Scratch floats of one layer's weight and bias gradients over M output pixels.
size_t layer_partial_floats(int l, int64_t M) {
  (void)M;
  const size_t cin = l == 0 ? 8 : kCin[l];         // the first layer runs on 8 padded channels
  const size_t ch = wgrad_chunks(l == 0 ? 8 : kCin[l]);
  return ch * kCout[l] * (9 * cin + 1);                // weight, then bias partial sums
}

// Scratch floats the weight and bias gradients of every layer of the network need at batch B.
size_t grad_partial_floats(int B) {
  static const int hin[5] = {256, 256, 128, 128, 64};
  size_t most = (size_t)((B + kHeadImgs - 1) / kHeadImgs) * kHeadParams;
  for (int l = 0; l < 5; ++l) {
    const int64_t ho = hin[l] / kStride[l];
    most = std::max(most, layer_partial_floats(l, (int64_t)B * ho * ho));
  }
  return most;
}

// Tensor maps of the weight-gradient kernel's operands: G (COUT, Ho, Ho, B) in boxes of 8 co x 64
// pixels x WT_ROWS rows; X (CIN, H, H, B) in boxes of 8 ci x NP entries x XROWS rows, or for S = 2
// the column-parity view (CIN, 2, H/2, H, B), its rows traversed with a stride of 2 for one tap row.
template <int CIN, int COUT, int S, int DYB>
int wgrad_maps(const __nv_bfloat16* G, const __nv_bfloat16* in, int B, int H, CUtensorMap* gmap,
               CUtensorMap* xmap) {
  const PFN_cuTensorMapEncodeTiled_v12000 encode = tensor_map_encoder();
  if (!encode) return GFH_ERR_CUDA;
  const cuuint64_t e = 2, Ho = (cuuint64_t)(H / S);
  constexpr int NP = WgradTc<CIN, COUT, S, DYB>::NP, XROWS = WgradTc<CIN, COUT, S, DYB>::XROWS;
  {
    const cuuint64_t dims[4] = {(cuuint64_t)COUT, Ho, Ho, (cuuint64_t)B};
    const cuuint64_t strides[3] = {COUT * e, Ho * COUT * e, Ho * Ho * COUT * e};
    const cuuint32_t box[4] = {8, 64, WT_ROWS, 1}, es[4] = {1, 1, 1, 1};
    if (encode(gmap, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 4, (void*)G, dims, strides, box, es,
               CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE,
               CU_TENSOR_MAP_L2_PROMOTION_L2_128B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) != CUDA_SUCCESS)
      return GFH_ERR_CUDA;
  }
  const cuuint64_t h = (cuuint64_t)H;
  CUresult r;
  if (S == 1) {
    const cuuint64_t dims[4] = {(cuuint64_t)CIN, h, h, (cuuint64_t)B};
    const cuuint64_t strides[3] = {CIN * e, h * CIN * e, h * h * CIN * e};
    const cuuint32_t box[4] = {8, (cuuint32_t)NP, XROWS, 1}, es[4] = {1, 1, 1, 1};
    r = encode(xmap, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 4, (void*)in, dims, strides, box, es,
               CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE,
               CU_TENSOR_MAP_L2_PROMOTION_L2_128B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  } else {
    const cuuint64_t dims[5] = {(cuuint64_t)CIN, 2, h / 2, h, (cuuint64_t)B};
    const cuuint64_t strides[4] = {CIN * e, 2 * CIN * e, h * CIN * e, h * h * CIN * e};
    // one tap row: rows 2 (y0 + r) + dy - 1 (stride 2); all tap rows: XROWS consecutive rows
    const cuuint32_t rstride = DYB == 1 ? 2 : 1;
    const cuuint32_t box[5] = {8, 1, (cuuint32_t)NP, (cuuint32_t)XROWS * rstride, 1},
                     es[5] = {1, 1, 1, rstride, 1};
    r = encode(xmap, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 5, (void*)in, dims, strides, box, es,
               CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE,
               CU_TENSOR_MAP_L2_PROMOTION_L2_128B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  }
  return r == CUDA_SUCCESS ? GFH_OK : GFH_ERR_CUDA;
}

// Launch of k_wgrad_tma over the layer's pixel chunks (x 3 tap rows for DYB = 1): weight partial
// sums to part [chunks][COUT][9][CIN], bias partial sums after them ([chunks][COUT]).
template <int CIN, int COUT, int S>
int wgrad_launch(const __nv_bfloat16* G, const __nv_bfloat16* in, int B, int H, float* part,
                 cudaStream_t st, unsigned int* flag) {
  constexpr int DYB = wgrad_dyb(CIN), chunks = wgrad_chunks(CIN);
  if ((H / S) % 64 || H % S) return GFH_ERR_ARG;
  alignas(64) CUtensorMap gmap, xmap;
  const int rc = wgrad_maps<CIN, COUT, S, DYB>(G, in, B, H, &gmap, &xmap);
  if (rc) return rc;
  constexpr int smem = WgradTc<CIN, COUT, S, DYB>::SMEM;
  static_assert(smem <= (int)kMaxSmemBytes - 4096, "weight-gradient stages fit in shared memory");
  auto fn = k_wgrad_tma<CIN, COUT, S, DYB>;
  GFH_CUDA_TRY(cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, smem));
  float* bias_part = part + (size_t)chunks * COUT * 9 * CIN;
  fn<<<dim3(chunks, DYB == 3 ? 1 : 3), WT_THREADS, smem, st>>>(gmap, xmap, part, bias_part, B, H,
                                                                chunks, flag);
  GFH_CUDA_TRY(cudaGetLastError());
  return GFH_OK;
}

// Weight gradient on tcgen05 (k_wgrad_tma) added into dw and bias gradient into db, from the
// gradient in the pre-activation G (masked); output rows and columns a multiple of 64.
template <int CIN, int COUT, int S>
int conv_wgrad_tc(const __nv_bfloat16* G, const __nv_bfloat16* in, float* dw, float* db, int B,
                  int H, float* part, cudaStream_t st, unsigned int* flag) {
  const int rc = wgrad_launch<CIN, COUT, S>(G, in, B, H, part, st, flag);
  if (rc) return rc;
  const int n = COUT * 9 * CIN, chunks = wgrad_chunks(CIN);
  k_sum_chunks<<<(n + 255) / 256, 256, 0, st>>>(part, chunks, n, dw);
  GFH_CUDA_TRY(cudaGetLastError());
  k_sum_chunks<<<1, 64, 0, st>>>(part + (size_t)chunks * n, chunks, COUT, db);
  GFH_CUDA_TRY(cudaGetLastError());
  return GFH_OK;
}

// First layer (2 input channels) weight and bias gradients, added into dw and db, from G1 (the
// gradient in layer 1's pre-activation, stored masked); img8 receives (padded = false) or already
// holds (padded = true, as the forward left it) the image padded to 8 channels, B H H x 8 bf16.
int conv1_wgrad(const __nv_bfloat16* g1, const __nv_bfloat16* in, __nv_bfloat16* img8, float* dw,
                float* db, int B, int H, float* part, cudaStream_t st, unsigned int* flag,
                bool padded) {
  const int64_t P1 = (int64_t)B * H * H;
  if (!padded) {
    k_pad_channels<<<(unsigned)((P1 + 255) / 256), 256, 0, st>>>((const uint32_t*)in, (int4*)img8, P1);
    GFH_CUDA_TRY(cudaGetLastError());
  }
  const int rc = wgrad_launch<8, 32, 1>(g1, img8, B, H, part, st, flag);
  if (rc) return rc;
  k_sum_chunks_l1<<<(576 + 255) / 256, 256, 0, st>>>(part, WT_CHUNKS1, dw);
  GFH_CUDA_TRY(cudaGetLastError());
  k_sum_chunks<<<1, 64, 0, st>>>(part + (size_t)WT_CHUNKS1 * 32 * 9 * 8, WT_CHUNKS1, 32, db);
  GFH_CUDA_TRY(cudaGetLastError());
  return GFH_OK;
}

}  // namespace

// ---- the network object -------------------------------------------------------------------------

struct gfh_cnn {
  gfh_ctx* ctx = nullptr;
  int max_batch = 0;
  Layout L{};
  int64_t step = 0;
  void* buf = nullptr;
  float *w = nullptr, *gw = nullptr, *m = nullptr, *v = nullptr;   // fp32 params, grads, Adam
  __nv_bfloat16* wb[5] = {};                                       // bf16 copies of W1..W5
  __nv_bfloat16* act[6] = {};                                      // a0 (input copy) .. a5
  __nv_bfloat16* dact[6] = {};                                     // d a1 .. d a5 (index 1..5)
  float *pooled = nullptr, *logits = nullptr, *dlogits = nullptr, *loss = nullptr;
  float* part = nullptr;                                           // gradient partial sums
  __nv_bfloat16* img8 = nullptr;                                   // input padded to 8 channels
  uint32_t* mbits[5] = {};                                         // ReLU masks of a1 .. a4 (1..4)
};

namespace {

size_t act_elems(int l, int B) {   // activation l (0 = input) element count
  static const int hw[6] = {256, 256, 128, 128, 64, 64};
  static const int ch[6] = {2, 32, 32, 64, 64, 64};
  return (size_t)B * hw[l] * hw[l] * ch[l];
}

void init_params(float* h, const Layout& L, uint64_t seed) {
  std::memset(h, 0, L.total * sizeof(float));
  uint64_t ctr = 0;
  auto uni = [&]() {   // uniform in [-1, 1) from the same splitmix64 finaliser
    return (double)(gfh_mix64(seed ^ (ctr++ * 0xD1B54A32D192ED03ull)) >> 11) * (1.0 / 9007199254740992.0) * 2.0 - 1.0;
  };
  for (int l = 0; l < 5; ++l) {
    const double bound = std::sqrt(6.0 / (9.0 * kCin[l]));   // He-uniform for ReLU
    for (int e = 0; e < kCout[l] * 9 * kCin[l]; ++e) h[L.w[l] + e] = (float)(bound * uni());
  }
  const double bh = std::sqrt(3.0 / (3.0 * 64.0));
  for (int e = 0; e < 64 * 3 * 64; ++e) h[L.wh + e] = (float)(bh * uni());
}

int refresh_bf16(gfh_cnn* n) {
  for (int l = 0; l < 5; ++l) {
    const int64_t cnt = (int64_t)kCout[l] * 9 * kCin[l];
    k_to_bf16<<<(unsigned)((cnt + 255) / 256), 256, 0, n->ctx->stream>>>(n->w + n->L.w[l], n->wb[l], cnt);
    GFH_CUDA_TRY(cudaGetLastError());
  }
  return GFH_OK;
}

// Forward pass; `masks`: also store the ReLU masks of a1 .. a4 (bits per channel) for the backward.
int forward(gfh_cnn* n, const __nv_bfloat16* img, int B, bool masks) {
  cudaStream_t st = n->ctx->stream;
  const int sms = n->ctx->num_sms;
  const Layout& L = n->L;
  unsigned int* flag = n->ctx->d_flag;
  uint32_t* const* mb = n->mbits;
  int rc = conv1_fwd(img, n->img8, n->wb[0], n->w + L.b[0], masks ? mb[1] : nullptr, n->act[1],
                     B, 256, sms, st, flag);
  if (!rc) rc = conv_fwd<32, 32, 2>(n->act[1], n->wb[1], n->w + L.b[1], nullptr, masks ? mb[2] : nullptr,
                                    n->act[2], B, 256, sms, st, flag);
  if (!rc) rc = conv_fwd<32, 64, 1>(n->act[2], n->wb[2], n->w + L.b[2], nullptr, masks ? mb[3] : nullptr,
                                    n->act[3], B, 128, sms, st, flag);
  if (!rc) rc = conv_fwd<64, 64, 2>(n->act[3], n->wb[3], n->w + L.b[3], nullptr, masks ? mb[4] : nullptr,
                                    n->act[4], B, 128, sms, st, flag);
  if (!rc) rc = conv_fwd<64, 64, 1>(n->act[4], n->wb[4], n->w + L.b[4], nullptr, nullptr, n->act[5],
                                    B, 64, sms, st, flag);
  if (rc) return rc;
  k_pool<<<(B * 4096 + 255) / 256, 256, 0, st>>>(n->act[5], n->pooled, B);
  k_head_fwd<<<dim3(kTiles / kHeadKtPerBlock, B), 256, 0, st>>>(n->pooled, n->w + L.wh, n->w + L.bh,
                                                                n->w + L.bnull, n->logits);
  GFH_CUDA_TRY(cudaGetLastError());
  return GFH_OK;
}

// Gradients of the mean loss into n->gw (zeroed first); per-sample losses in n->loss.
int backward(gfh_cnn* n, const __nv_bfloat16* img, const int32_t* labels, int B) {
  cudaStream_t st = n->ctx->stream;
  unsigned int* flag = n->ctx->d_flag;
  const int sms = n->ctx->num_sms;
  const Layout& L = n->L;
  GFH_CUDA_TRY(cudaMemsetAsync(n->gw, 0, L.total * sizeof(float), st));
  k_softmax_ce<<<B, 256, 0, st>>>(n->logits, labels, n->dlogits, n->loss, B);
  const int hchunks = (B + kHeadImgs - 1) / kHeadImgs;
  k_head_wgrad<<<dim3((kHeadParams + 255) / 256, hchunks), 256, 0, st>>>(n->dlogits, n->pooled, n->part, B);
  k_sum_chunks<<<(kHeadParams + 255) / 256, 256, 0, st>>>(n->part, hchunks, kHeadParams, n->gw + L.wh);
  k_head_dgrad<<<(B * 4096 + 255) / 256, 256, 0, st>>>(n->dlogits, n->w + L.wh, n->act[5], n->dact[5], B);
  GFH_CUDA_TRY(cudaGetLastError());
  int rc = conv_wgrad_tc<64, 64, 1>(n->dact[5], n->act[4], n->gw + L.w[4], n->gw + L.b[4], B, 64, n->part, st, flag);
  if (!rc) rc = conv_fwd<64, 64, 1, 1>(n->dact[5], n->wb[4], nullptr, n->mbits[4], nullptr, n->dact[4], B, 64, sms, st, flag);
  if (!rc) rc = conv_wgrad_tc<64, 64, 2>(n->dact[4], n->act[3], n->gw + L.w[3], n->gw + L.b[3], B, 128, n->part, st, flag);
  if (!rc) rc = conv_fwd<64, 64, 1, 2>(n->dact[4], n->wb[3], nullptr, n->mbits[3], nullptr, n->dact[3], B, 128, sms, st, flag);
  if (!rc) rc = conv_wgrad_tc<32, 64, 1>(n->dact[3], n->act[2], n->gw + L.w[2], n->gw + L.b[2], B, 128, n->part, st, flag);
  if (!rc) rc = conv_fwd<64, 32, 1, 1>(n->dact[3], n->wb[2], nullptr, n->mbits[2], nullptr, n->dact[2], B, 128, sms, st, flag);
  if (!rc) rc = conv_wgrad_tc<32, 32, 2>(n->dact[2], n->act[1], n->gw + L.w[1], n->gw + L.b[1], B, 256, n->part, st, flag);
  if (!rc) rc = conv_fwd<32, 32, 1, 2>(n->dact[2], n->wb[1], nullptr, n->mbits[1], nullptr, n->dact[1], B, 256, sms, st, flag);
  if (rc) return rc;
  return conv1_wgrad(n->dact[1], img, n->img8, n->gw + L.w[0], n->gw + L.b[0], B, kImg, n->part, st,
                     flag, true);
}

}  // namespace

extern "C" int gfh_cnn_create(gfh_ctx* ctx, int32_t max_batch, uint64_t seed, gfh_cnn** out) {
  if (!ctx || !out || max_batch < 1 || max_batch > 4096) return GFH_ERR_ARG;
  *out = nullptr;
  gfh_cnn* n = new (std::nothrow) gfh_cnn();
  if (!n) return GFH_ERR_NOMEM;
  n->ctx = ctx;
  n->max_batch = max_batch;
  n->L = make_layout();
  const int B = max_batch;
  size_t off = 0;
  auto take = [&](size_t bytes) { size_t o = off; off = (off + bytes + 255) / 256 * 256; return o; };
  const size_t o_w = take(n->L.total * 4), o_gw = take(n->L.total * 4), o_m = take(n->L.total * 4),
               o_v = take(n->L.total * 4);
  size_t o_wb[5], o_act[6], o_dact[6];
  for (int l = 0; l < 5; ++l) o_wb[l] = take((size_t)kCout[l] * 9 * kCin[l] * 2);
  for (int l = 1; l < 6; ++l) { o_act[l] = take(act_elems(l, B) * 2); o_dact[l] = take(act_elems(l, B) * 2); }
  const size_t o_pool = take((size_t)B * 4096 * 4), o_log = take((size_t)B * kClasses * 4),
               o_dlog = take((size_t)B * kClasses * 4), o_loss = take((size_t)B * 4),
               o_part = take(grad_partial_floats(B) * 4),
               o_img8 = take((size_t)B * kImg * kImg * 16);
  size_t o_mb[5] = {};
  for (int l = 1; l < 5; ++l) o_mb[l] = take(act_elems(l, B) / 8);   // one bit per element
  if (cudaSetDevice(ctx->device) != cudaSuccess) { delete n; return GFH_ERR_CUDA; }
  if (cudaMalloc(&n->buf, off) != cudaSuccess) { delete n; return GFH_ERR_NOMEM; }
  char* base = (char*)n->buf;
  n->w = (float*)(base + o_w); n->gw = (float*)(base + o_gw);
  n->m = (float*)(base + o_m); n->v = (float*)(base + o_v);
  for (int l = 0; l < 5; ++l) n->wb[l] = (__nv_bfloat16*)(base + o_wb[l]);
  for (int l = 1; l < 6; ++l) {
    n->act[l] = (__nv_bfloat16*)(base + o_act[l]);
    n->dact[l] = (__nv_bfloat16*)(base + o_dact[l]);
  }
  n->pooled = (float*)(base + o_pool); n->logits = (float*)(base + o_log);
  n->dlogits = (float*)(base + o_dlog); n->loss = (float*)(base + o_loss);
  n->part = (float*)(base + o_part);
  n->img8 = (__nv_bfloat16*)(base + o_img8);
  for (int l = 1; l < 5; ++l) n->mbits[l] = (uint32_t*)(base + o_mb[l]);
  float* h = new (std::nothrow) float[n->L.total];
  if (!h) { cudaFree(n->buf); delete n; return GFH_ERR_NOMEM; }
  init_params(h, n->L, seed);
  cudaError_t e = cudaMemcpy(n->w, h, n->L.total * 4, cudaMemcpyHostToDevice);
  delete[] h;
  if (e == cudaSuccess) e = cudaMemset(n->m, 0, n->L.total * 4);
  if (e == cudaSuccess) e = cudaMemset(n->v, 0, n->L.total * 4);
  if (e != cudaSuccess || refresh_bf16(n) != GFH_OK || cudaStreamSynchronize(ctx->stream) != cudaSuccess) {
    cudaFree(n->buf);
    delete n;
    return GFH_ERR_CUDA;
  }
  *out = n;
  return GFH_OK;
}

extern "C" int gfh_cnn_destroy(gfh_cnn* n) {
  if (!n) return GFH_OK;
  cudaSetDevice(n->ctx->device);
  if (n->ctx->stream) cudaStreamSynchronize(n->ctx->stream);
  if (n->buf) cudaFree(n->buf);
  delete n;
  return GFH_OK;
}

extern "C" int64_t gfh_cnn_param_count(const gfh_cnn* n) { return n ? (int64_t)n->L.total : -1; }

extern "C" int gfh_cnn_get_params(gfh_cnn* n, float* h_params, float* h_grads) {
  if (!n) return GFH_ERR_ARG;
  GFH_CUDA_TRY(cudaStreamSynchronize(n->ctx->stream));
  if (h_params) GFH_CUDA_TRY(cudaMemcpy(h_params, n->w, n->L.total * 4, cudaMemcpyDeviceToHost));
  if (h_grads) GFH_CUDA_TRY(cudaMemcpy(h_grads, n->gw, n->L.total * 4, cudaMemcpyDeviceToHost));
  return GFH_OK;
}

extern "C" int gfh_cnn_set_params(gfh_cnn* n, const float* h_params) {
  if (!n || !h_params) return GFH_ERR_ARG;
  GFH_CUDA_TRY(cudaStreamSynchronize(n->ctx->stream));
  GFH_CUDA_TRY(cudaMemcpy(n->w, h_params, n->L.total * 4, cudaMemcpyHostToDevice));
  GFH_CUDA_TRY(cudaMemset(n->m, 0, n->L.total * 4));
  GFH_CUDA_TRY(cudaMemset(n->v, 0, n->L.total * 4));
  n->step = 0;
  return refresh_bf16(n);
}

extern "C" int gfh_cnn_get_state(gfh_cnn* n, float* h_params, float* h_m, float* h_v,
                                 int64_t* h_step) {
  if (!n) return GFH_ERR_ARG;
  GFH_CUDA_TRY(cudaSetDevice(n->ctx->device));
  GFH_CUDA_TRY(cudaStreamSynchronize(n->ctx->stream));
  const size_t bytes = n->L.total * 4;
  if (h_params) GFH_CUDA_TRY(cudaMemcpy(h_params, n->w, bytes, cudaMemcpyDeviceToHost));
  if (h_m) GFH_CUDA_TRY(cudaMemcpy(h_m, n->m, bytes, cudaMemcpyDeviceToHost));
  if (h_v) GFH_CUDA_TRY(cudaMemcpy(h_v, n->v, bytes, cudaMemcpyDeviceToHost));
  if (h_step) *h_step = n->step;
  return GFH_OK;
}

extern "C" int gfh_cnn_set_state(gfh_cnn* n, const float* h_params, const float* h_m,
                                 const float* h_v, int64_t step) {
  if (!n || !h_params || !h_m || !h_v || step < 0) return GFH_ERR_ARG;
  GFH_CUDA_TRY(cudaSetDevice(n->ctx->device));
  GFH_CUDA_TRY(cudaStreamSynchronize(n->ctx->stream));
  const size_t bytes = n->L.total * 4;
  GFH_CUDA_TRY(cudaMemcpy(n->w, h_params, bytes, cudaMemcpyHostToDevice));
  GFH_CUDA_TRY(cudaMemcpy(n->m, h_m, bytes, cudaMemcpyHostToDevice));
  GFH_CUDA_TRY(cudaMemcpy(n->v, h_v, bytes, cudaMemcpyHostToDevice));
  n->step = step;
  int rc = refresh_bf16(n);
  if (!rc) GFH_CUDA_TRY(cudaStreamSynchronize(n->ctx->stream));
  return rc;
}

extern "C" int gfh_cnn_read_tensor(gfh_cnn* n, int32_t which, int32_t batch, void* h_out,
                                   int64_t bytes) {
  if (!n || !h_out || batch < 1 || batch > n->max_batch) return GFH_ERR_ARG;
  const void* src = nullptr;
  size_t need = 0;
  if (which >= GFH_CNN_ACT && which <= GFH_CNN_ACT + 5 && which != GFH_CNN_ACT) {
    src = n->act[which - GFH_CNN_ACT];
    need = act_elems(which - GFH_CNN_ACT, batch) * 2;
  } else if (which > GFH_CNN_DACT && which <= GFH_CNN_DACT + 5) {
    src = n->dact[which - GFH_CNN_DACT];
    need = act_elems(which - GFH_CNN_DACT, batch) * 2;
  } else if (which >= GFH_CNN_WBF16 && which < GFH_CNN_WBF16 + 5) {
    const int l = which - GFH_CNN_WBF16;
    src = n->wb[l];
    need = (size_t)kCout[l] * 9 * kCin[l] * 2;
  } else if (which == GFH_CNN_POOLED) {
    src = n->pooled;
    need = (size_t)batch * 4096 * 4;
  } else if (which == GFH_CNN_LOGITS || which == GFH_CNN_DLOGITS) {
    src = which == GFH_CNN_LOGITS ? n->logits : n->dlogits;
    need = (size_t)batch * kClasses * 4;
  } else if (which == GFH_CNN_LOSS) {
    src = n->loss;
    need = (size_t)batch * 4;
  } else {
    return GFH_ERR_ARG;
  }
  if (bytes < (int64_t)need) return GFH_ERR_SIZE;
  GFH_CUDA_TRY(cudaSetDevice(n->ctx->device));
  GFH_CUDA_TRY(cudaStreamSynchronize(n->ctx->stream));
  GFH_CUDA_TRY(cudaMemcpy(h_out, src, need, cudaMemcpyDeviceToHost));
  return GFH_OK;
}

extern "C" int gfh_cnn_forward(gfh_cnn* n, const void* d_images, int32_t batch, float* d_logits) {
  if (!n || !d_images || batch < 1 || batch > n->max_batch) return GFH_ERR_ARG;
  GFH_CUDA_TRY(cudaSetDevice(n->ctx->device));
  int rc = forward(n, (const __nv_bfloat16*)d_images, batch, false);
  if (rc) return rc;
  if (d_logits)
    GFH_CUDA_TRY(cudaMemcpyAsync(d_logits, n->logits, (size_t)batch * kClasses * 4,
                                 cudaMemcpyDeviceToDevice, n->ctx->stream));
  return GFH_OK;
}

extern "C" int gfh_cnn_gradients(gfh_cnn* n, const void* d_images, const int32_t* d_labels,
                                 int32_t batch, float* h_loss) {
  if (!n || !d_images || !d_labels || batch < 1 || batch > n->max_batch) return GFH_ERR_ARG;
  GFH_CUDA_TRY(cudaSetDevice(n->ctx->device));
  int rc = forward(n, (const __nv_bfloat16*)d_images, batch, true);
  if (!rc) rc = backward(n, (const __nv_bfloat16*)d_images, d_labels, batch);
  if (rc) return rc;
  if (h_loss) {
    float* tmp = new (std::nothrow) float[batch];
    if (!tmp) return GFH_ERR_NOMEM;
    cudaError_t e = cudaMemcpyAsync(tmp, n->loss, (size_t)batch * 4, cudaMemcpyDeviceToHost, n->ctx->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(n->ctx->stream);
    double s = 0.0;
    for (int b = 0; b < batch; ++b) s += tmp[b];
    delete[] tmp;
    if (e != cudaSuccess) return GFH_ERR_CUDA;
    *h_loss = (float)(s / batch);
  }
  return GFH_OK;
}

extern "C" int gfh_cnn_train_step(gfh_cnn* n, const void* d_images, const int32_t* d_labels,
                                  int32_t batch, float lr, float weight_decay, float* h_loss) {
  int rc = gfh_cnn_gradients(n, d_images, d_labels, batch, h_loss);
  if (rc) return rc;
  n->step += 1;
  const float b1 = 0.9f, b2 = 0.999f;
  const float c1 = 1.f - std::pow(b1, (float)n->step), c2 = 1.f - std::pow(b2, (float)n->step);
  const int64_t cnt = (int64_t)n->L.total;
  k_adamw<<<(unsigned)((cnt + 255) / 256), 256, 0, n->ctx->stream>>>(n->w, n->gw, n->m, n->v, cnt, lr,
                                                                    b1, b2, 1e-8f, weight_decay, c1, c2);
  GFH_CUDA_TRY(cudaGetLastError());
  return refresh_bf16(n);
}

extern "C" int gfh_synth_images(gfh_ctx* ctx, uint64_t seed, int64_t sample0, int32_t batch,
                                int32_t n_fft, int32_t bin_lo, int32_t bin_hi, uint32_t p_noise24,
                                const uint32_t* d_p_track24, const int32_t* d_tracks,
                                const float* d_nplane, void* d_images) {
  if (!ctx || batch < 1 || n_fft < kImg || bin_lo < 0 || bin_hi < bin_lo ||
      bin_hi - bin_lo + 1 < kImg || !d_p_track24 || !d_tracks || !d_nplane || !d_images ||
      batch > 65535)
    return GFH_ERR_ARG;
  GFH_CUDA_TRY(cudaSetDevice(ctx->device));
  dim3 grid((kImg * kImg + 255) / 256, batch);
  k_synth_images<<<grid, 256, 0, ctx->stream>>>(seed, sample0, n_fft, bin_lo, bin_hi - bin_lo + 1,
                                                p_noise24, d_p_track24, d_tracks, d_nplane,
                                                ctx->d_log1p, (uint32_t*)d_images);
  GFH_CUDA_TRY(cudaGetLastError());
  return GFH_OK;
}

extern "C" int gfh_peaks_to_images(gfh_ctx* ctx, const gfh_peaks* peaks, int32_t n_fft,
                                   int32_t bin_lo, int32_t bin_hi, const float* d_nplane,
                                   void* d_images) {
  if (!ctx || !peaks || !peaks->offsets || peaks->n_lists < 1 || peaks->n_lists > 65535 ||
      !peaks->fft_idx || !peaks->bin || n_fft < kImg || n_fft >= (1 << 24) || bin_lo < 0 ||
      bin_hi < bin_lo || bin_hi - bin_lo + 1 < kImg || bin_hi - bin_lo + 1 >= (1 << 24) ||
      !d_nplane || !d_images)
    return GFH_ERR_ARG;
  GFH_CUDA_TRY(cudaSetDevice(ctx->device));
  const int L = peaks->n_lists;
  uint32_t* img = (uint32_t*)d_images;
  GFH_CUDA_TRY(cudaMemsetAsync(img, 0, (size_t)L * kImg * kImg * 4, ctx->stream));
  const int gx = std::max(1, std::min(64, ctx->num_sms * 8 / L));
  k_image_count<<<dim3(gx, L), 256, 0, ctx->stream>>>(peaks->fft_idx, peaks->bin, peaks->offsets,
                                                       n_fft, bin_lo, bin_hi - bin_lo + 1, img,
                                                       ctx->d_flag);
  GFH_CUDA_TRY(cudaGetLastError());
  k_image_finish<<<dim3(kImg * kImg / 256, L), 256, 0, ctx->stream>>>(img, d_nplane, ctx->d_log1p);
  GFH_CUDA_TRY(cudaGetLastError());
  return GFH_OK;
}

extern "C" int gfh_propose_tiles(gfh_ctx* ctx, const float* d_logits, int32_t batch,
                                 const float* d_gain, int32_t k, float tau, int32_t* d_top,
                                 float* d_resid, int32_t* d_full) {
  if (!ctx || !d_logits || !d_gain || !d_top || !d_resid || batch < 1 || k < 1 ||
      k > kTiles * kTiles || !(tau == tau))
    return GFH_ERR_ARG;
  GFH_CUDA_TRY(cudaSetDevice(ctx->device));
  k_propose<<<batch, 1024, 0, ctx->stream>>>(d_logits, d_gain, k, tau, d_top, d_resid, d_full);
  GFH_CUDA_TRY(cudaGetLastError());
  return GFH_OK;
}

extern "C" int gfh_line_scores(gfh_ctx* ctx, const void* d_images, int32_t batch, int32_t n_k,
                               int32_t n_bins, float beta, float det_a, float det_c,
                               float* d_scores, float* d_logits) {
  if (!ctx || !d_images || !d_logits || batch < 1 || batch > 65535 || n_k < 1 || n_bins < kImg ||
      !(beta >= 0.f) || !(det_a == det_a) || !(det_c == det_c))
    return GFH_ERR_ARG;
  GFH_CUDA_TRY(cudaSetDevice(ctx->device));
  const int smem = kImg * kImg * 2 + kTiles * kImg * 4;
  GFH_CUDA_TRY(cudaFuncSetAttribute(k_line_scores, cudaFuncAttributeMaxDynamicSharedMemorySize, smem));
  k_line_scores<<<batch, 1024, smem, ctx->stream>>>((const uint32_t*)d_images, n_k, n_bins, beta,
                                                    det_a, det_c, d_scores, d_logits);
  GFH_CUDA_TRY(cudaGetLastError());
  return GFH_OK;
}

extern "C" int gfh_wait_check(gfh_ctx* ctx, int64_t cycles) {
  if (!ctx || cycles < 0 || cycles > 4000000000ll) return GFH_ERR_ARG;
  GFH_CUDA_TRY(cudaSetDevice(ctx->device));
  k_wait_unsignalled<<<1, 32, 0, ctx->stream>>>((long long)cycles, ctx->d_flag);
  GFH_CUDA_TRY(cudaGetLastError());
  return GFH_OK;
}

// One 3x3 layer in isolation (for tests): mode 0 forward, 1 input gradient, 2 weight gradient.
extern "C" int gfh_conv3x3(gfh_ctx* ctx, int32_t mode, int32_t cin, int32_t cout, int32_t stride,
                           int32_t batch, int32_t h, const void* d_in, const void* d_w,
                           const float* d_bias, const void* d_out, const void* d_dout, void* d_res,
                           float* d_db) {
  if (!ctx || batch < 1 || h < 16 || h % 16) return GFH_ERR_ARG;
  GFH_CUDA_TRY(cudaSetDevice(ctx->device));
  const int sms = ctx->num_sms;
  cudaStream_t st = ctx->stream;
  const auto* in = (const __nv_bfloat16*)d_in;
  const auto* w = (const __nv_bfloat16*)d_w;
  const auto* out = (const __nv_bfloat16*)d_out;
  const auto* dout = (const __nv_bfloat16*)d_dout;
  float* part = nullptr;
  size_t part_bytes = 0;
  if (mode == 0 && cin == 2) {   // the image padded to 8 channels in the context scratch
    const int rc = ensure_scratch(ctx, (size_t)batch * h * h * 16);
    if (rc) return rc;
  }
  if (mode == 1) {   // the masked gradient in the context scratch
    const int rc = ensure_scratch(ctx, (size_t)batch * (h / stride) * (h / stride) * cout * 2);
    if (rc) return rc;
  }
  if (mode == 2) {   // partial sums in the context scratch, then (L2-L5) the masked gradient
    int l = -1;
    for (int q = 0; q < 5; ++q)
      if (kCin[q] == cin && kCout[q] == cout && kStride[q] == stride) l = q;
    if (l < 0) return GFH_ERR_ARG;
    const int64_t ho = h / stride;
    part_bytes = (layer_partial_floats(l, (int64_t)batch * ho * ho) * 4 + 255) / 256 * 256;
    // then the masked gradient, and for the first layer the input padded to 8 channels
    const int rc = ensure_scratch(ctx, part_bytes + (size_t)batch * ho * ho * cout * 2 +
                                           (l == 0 ? (size_t)batch * h * h * 16 : 0));
    if (rc) return rc;
    part = (float*)ctx->pm_buf;
  }
#define GFH_CONV_CASE(CI, CO, S)                                                                   \
  if (cin == CI && cout == CO && stride == S) {                                                    \
    if (mode == 0) return conv_fwd<CI, CO, S>(in, w, d_bias, nullptr, nullptr, (__nv_bfloat16*)d_res, batch, h, sms, st, ctx->d_flag); \
    if (mode == 1) {                                                                               \
      const int64_t n_el = (int64_t)batch * (h / S) * (h / S) * CO;                                \
      __nv_bfloat16* g = (__nv_bfloat16*)ctx->pm_buf;                                              \
      k_mask_grad<<<(unsigned)((n_el + 255) / 256), 256, 0, st>>>(dout, out, g, n_el);              \
      GFH_CUDA_TRY(cudaGetLastError());                                                            \
      return conv_fwd<CO, CI, 1, S == 1 ? 1 : 2>(g, w, nullptr, nullptr, nullptr, (__nv_bfloat16*)d_res, \
                                                 batch, h, sms, st, ctx->d_flag);                  \
    }                                                                                              \
    if (mode == 2) {                                                                               \
      const int64_t n_el = (int64_t)batch * (h / S) * (h / S) * CO;                                \
      __nv_bfloat16* g = (__nv_bfloat16*)((char*)ctx->pm_buf + part_bytes);                       \
      k_mask_grad<<<(unsigned)((n_el + 255) / 256), 256, 0, st>>>(dout, out, g, n_el);              \
      GFH_CUDA_TRY(cudaGetLastError());                                                            \
      return conv_wgrad_tc<CI, CO, S>(g, in, (float*)d_res, d_db, batch, h, part, st, ctx->d_flag); \
    }                                                                                              \
    return GFH_ERR_ARG;                                                                            \
  }
  if (cin == 2 && cout == 32 && stride == 1) {                      // first layer: no input gradient
    if (mode == 0)
      return conv1_fwd(in, (__nv_bfloat16*)ctx->pm_buf, w, d_bias, nullptr, (__nv_bfloat16*)d_res,
                       batch, h, sms, st, ctx->d_flag);
    if (mode == 2) {
      const int64_t n_el = (int64_t)batch * h * h * 32;
      __nv_bfloat16* g = (__nv_bfloat16*)((char*)ctx->pm_buf + part_bytes);
      __nv_bfloat16* img8 = g + n_el;
      k_mask_grad<<<(unsigned)((n_el + 255) / 256), 256, 0, st>>>(dout, out, g, n_el);
      GFH_CUDA_TRY(cudaGetLastError());
      return conv1_wgrad(g, in, img8, (float*)d_res, d_db, batch, h, part, st, ctx->d_flag, false);
    }
    return GFH_ERR_ARG;
  }
  GFH_CONV_CASE(32, 32, 2)
  GFH_CONV_CASE(32, 64, 1)
  GFH_CONV_CASE(64, 64, 2)
  GFH_CONV_CASE(64, 64, 1)
#undef GFH_CONV_CASE
  return GFH_ERR_ARG;
}
