// Peakmap (Sec. III) on sm_103a: interlaced short FFTs (cuFFT), equalisation by a clipped
// auto-regressive mean along frequency, threshold + local-maximum test, and compaction of the
// peaks into (fft_idx, bin) lists sorted by bin then FFT.
//
// The equaliser is one sequential recurrence per FFT.  A warp owns 32 FFTs (one per lane); tiles
// of 32 FFTs x 32 bins are staged through shared memory with coalesced loads and every lane walks
// its own spectrum.  Each step's peak decisions of the warp form one 32-bit ballot word, stored in
// a bin-major bit matrix that the compaction kernels turn into sorted lists.
#include <mutex>

#include "gfh_internal.h"

namespace {

constexpr float kArWeight = 0.0078125f;   // 2^-7
constexpr float kGain = 1.08942544f;      // float32(1 / (1 - exp(-2.5)))
constexpr float kClipGain = 2.72356367f;  // float32(2.5 / (1 - exp(-2.5)))
constexpr int kWarm = 128;

// Power of one spectrum bin from the input layout: the raw element (Raw) copied to shared memory,
// its source address, and the power computed from it.
struct PowerIn {
  using Raw = float;
  const float* p;
  int64_t ld;
  __device__ __forceinline__ const Raw* src(int64_t i, int64_t j) const { return p + i * ld + j; }
  __device__ __forceinline__ static float power(Raw v) { return v; }
};
struct ComplexIn {
  using Raw = float2;
  const float2* x;
  int64_t ld;
  __device__ __forceinline__ const Raw* src(int64_t i, int64_t j) const { return x + i * ld + j; }
  __device__ __forceinline__ static float power(Raw v) {
    return __fadd_rn(__fmul_rn(v.x, v.x), __fmul_rn(v.y, v.y));
  }
};
// Spectra of a band only: x [n_fft][ld] holds bins j0 .. j0 + ld - 1.
struct BandIn {
  using Raw = float2;
  const float2* x;
  int64_t ld;
  int64_t j0;
  __device__ __forceinline__ const Raw* src(int64_t i, int64_t j) const {
    return x + i * ld + (j - j0);
  }
  __device__ __forceinline__ static float power(Raw v) {
    return __fadd_rn(__fmul_rn(v.x, v.x), __fmul_rn(v.y, v.y));
  }
};

// Asynchronous copy of one raw element (4 or 8 bytes) to shared memory; ok = false fills zeros
// (the source is then not read).
template <class Raw>
__device__ __forceinline__ void eq_copy(Raw* dst, const Raw* src, bool ok) {
  const uint32_t d = (uint32_t)__cvta_generic_to_shared(dst);
  asm volatile("cp.async.ca.shared.global [%0], [%1], %2, %3;" ::"r"(d), "l"(src),
               "n"((int)sizeof(Raw)), "r"(ok ? (int)sizeof(Raw) : 0)
               : "memory");
}

// bits[(b - bin_lo) * n_words + w], bit l: FFT 32 w + l has a peak in bin b.
//
// One block of kEqWarps warps per 32 FFTs (lane l = FFT 32 w + l), over chunks of 32 bins:
//   warp 0      runs only the recurrence of chunk c (the mean each bin is divided by, then the
//               update: four dependent operations per bin, the one serial part) and leaves the
//               means in shared memory;
//   warps 1..H  copy chunk c + kEqDepth into a ring in shared memory (asynchronous copies, one
//               group per chunk, each helper its own rows), divide chunk c-1 (helper h takes bins
//               h-1, h-1+H, ...), meet at a named barrier, take the peak decisions of chunk c-1 one
//               bin late (bin b needs R at b+1, one ballot word per bin), then wait for their rows
//               of chunk c+1 and turn them into powers for the recurrence.
// Rings: kEqDepth + 1 raw tiles, three power tiles, two mean tiles, two equalised tiles; one block
// barrier per chunk.  The copies run kEqDepth chunks ahead so that memory latency stays off the
// recurrence, and a full chunk past the warm-up is one straight-line run of 32 updates, its loads
// issued ahead of the chain.
constexpr int kEqWarps = 16;
constexpr int kEqHelpers = kEqWarps - 1;
constexpr int kEqDepth = 4;
constexpr int kEqRing = kEqDepth + 1;

template <class In>
size_t eq_smem_bytes() { return (size_t)kEqRing * 32 * 32 * sizeof(typename In::Raw); }

template <class In>
__global__ void __launch_bounds__(32 * kEqWarps) k_equalise(In in, int n_fft, int bin_lo,
                                                            int bin_hi, float theta,
                                                            uint32_t* __restrict__ bits,
                                                            int n_words) {
  using Raw = typename In::Raw;
  extern __shared__ __align__(16) unsigned char eq_dyn[];
  Raw* raw = reinterpret_cast<Raw*>(eq_dyn);   // [kEqRing][32 ffts][32 bins]
  __shared__ float Pt[3][32][33];   // [chunk ring][fft][bin]
  __shared__ float Sm[2][32][33];   // [chunk ring][fft][bin]: mean each bin is divided by
  __shared__ float Rt[2][32][32];   // [chunk ring][bin][fft]: equalised values
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int gw = blockIdx.x;        // word index: FFTs 32 gw .. 32 gw + 31
  const int fft0 = gw * 32;
  const int my_fft = fft0 + lane;
  const int j0 = bin_lo - 1 - kWarm;    // first warm-up bin
  const int j_end = bin_hi + 1;         // last equalised bin
  const int n_chunks = (j_end - j0 + 32) / 32;
  constexpr int kRowsPerHelper = (32 + kEqHelpers - 1) / kEqHelpers;
  const int h = warp - 1;
  // helper: copy its rows of chunk x (zeros past the last FFT or bin), as one commit group
  auto issue = [&](int x) {
    if (x < n_chunks) {
      Raw* slot = raw + (x % kEqRing) * 32 * 32;
#pragma unroll
      for (int i = 0; i < kRowsPerHelper; ++i) {
        const int r = h + i * kEqHelpers;
        if (r < 32) {
          const int f = fft0 + r, j = j0 + 32 * x + lane;
          const bool ok = f < n_fft && j <= j_end;
          eq_copy(slot + r * 32 + lane, ok ? in.src(f, j) : in.src(0, j0), ok);
        }
      }
    }
    asm volatile("cp.async.commit_group;" ::: "memory");
  };
  // helper: its rows of chunk x, raw -> power tile
  auto convert = [&](int x) {
    if (x < n_chunks) {
      const Raw* slot = raw + (x % kEqRing) * 32 * 32;
#pragma unroll
      for (int i = 0; i < kRowsPerHelper; ++i) {
        const int r = h + i * kEqHelpers;
        if (r < 32) Pt[x % 3][r][lane] = In::power(slot[r * 32 + lane]);
      }
    }
  };
  if (warp > 0) {
    for (int x = 0; x < kEqDepth; ++x) issue(x);
    asm volatile("cp.async.wait_group %0;" ::"n"(kEqDepth - 1) : "memory");   // chunk 0
    convert(0);
  }
  __syncthreads();
  float S = 0.f;                        // warp 0: running mean of FFT my_fft
  for (int c = 0; c <= n_chunks; ++c) {
    if (warp == 0) {
      if (c < n_chunks) {
        const int cb = j0 + 32 * c;
        const int nq = min(32, j_end - cb + 1);
        const float* row = Pt[c % 3][lane];
        float* srow = Sm[c & 1][lane];
        if (nq == 32 && cb >= bin_lo - 1) {
          // a full chunk past the warm-up (all but a few): straight-line code, so the chunk's
          // loads and the P-only products run ahead of the chain of dependent updates
          float P[32];
#pragma unroll
          for (int q = 0; q < 32; ++q) P[q] = row[q];
#pragma unroll
          for (int q = 0; q < 32; ++q) {
            srow[q] = S;
            const float u = fminf(__fmul_rn(P[q], kGain), __fmul_rn(S, kClipGain));
            S = __fadd_rn(S, __fmul_rn(kArWeight, __fsub_rn(u, S)));
          }
        } else {
#pragma unroll
          for (int q = 0; q < 32; ++q) {
            if (q < nq) {
              const int j = cb + q;
              const float P = row[q];
              srow[q] = S;
              if (j < bin_lo - 1) {
                S = __fadd_rn(S, P);
                if (j == bin_lo - 2) S = __fmul_rn(S, 1.0f / kWarm);
              } else {
                const float u = fminf(__fmul_rn(P, kGain), __fmul_rn(S, kClipGain));
                S = __fadd_rn(S, __fmul_rn(kArWeight, __fsub_rn(u, S)));
              }
            }
          }
        }
      }
    } else {
      issue(c + kEqDepth);
      if (c >= 1) {
        const int cp = c - 1;
        const int cb = j0 + 32 * cp;
        const int nq = min(32, j_end - cb + 1);
        // equalised values of this helper's bins: R_j = P_j / S_(j-1)
        for (int q = h; q < nq; q += kEqHelpers)
          if (cb + q >= bin_lo - 1)
            Rt[cp & 1][q][lane] = __fdiv_rn(Pt[cp % 3][lane][q], Sm[cp & 1][lane][q]);
        asm volatile("bar.sync 1, %0;" ::"n"(32 * kEqHelpers));
        // decisions for bins b = cb + q - 1: neighbours b-1, b, b+1 (the first two may sit in
        // the previous chunk's tile)
        for (int q = h; q < nq; q += kEqHelpers) {
          const int b = cb + q - 1;
          if (b < bin_lo || b > bin_hi) continue;
          const float rl = q >= 2 ? Rt[cp & 1][q - 2][lane] : Rt[(cp + 1) & 1][q + 30][lane];
          const float rc = q >= 1 ? Rt[cp & 1][q - 1][lane] : Rt[(cp + 1) & 1][31][lane];
          const float rr = Rt[cp & 1][q][lane];
          const bool pk = my_fft < n_fft && rc > theta && rc > rl && rc > rr;
          const uint32_t word = __ballot_sync(0xffffffffu, pk);
          if (lane == 0) bits[(int64_t)(b - bin_lo) * n_words + gw] = word;
        }
      }
      asm volatile("cp.async.wait_group %0;" ::"n"(kEqDepth - 1) : "memory");   // chunk c+1
      convert(c + 1);
    }
    __syncthreads();
  }
  asm volatile("cp.async.wait_all;" ::: "memory");
}

// Launch of the equaliser with its dynamic shared memory (the raw ring; above the default 48 KB
// with the static tiles, so the attribute is raised once per device and input type).
template <class In>
cudaError_t launch_equalise(In in, int n_fft, int bin_lo, int bin_hi, float theta, uint32_t* bits,
                            int n_words, cudaStream_t st) {
  static std::mutex mu;
  static uint64_t done = 0;
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  const size_t dyn = eq_smem_bytes<In>();
  {
    std::lock_guard<std::mutex> lock(mu);
    if (dev < 0 || dev >= 64 || !(done >> dev & 1ull)) {
      e = cudaFuncSetAttribute(k_equalise<In>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                               (int)dyn);
      if (e != cudaSuccess) return e;
      if (dev >= 0 && dev < 64) done |= 1ull << dev;
    }
  }
  k_equalise<In><<<n_words, 32 * kEqWarps, dyn, st>>>(in, n_fft, bin_lo, bin_hi, theta, bits,
                                                     n_words);
  return cudaGetLastError();
}

// counts[b] = peaks in bin b (one warp per bin).
__global__ void k_count(const uint32_t* __restrict__ bits, int n_bins, int n_words,
                        int64_t* __restrict__ counts) {
  const int b = blockIdx.x * (blockDim.x / 32) + (threadIdx.x >> 5);
  const int lane = threadIdx.x & 31;
  if (b >= n_bins) return;
  int c = 0;
  for (int w = lane; w < n_words; w += 32) c += __popc(bits[(int64_t)b * n_words + w]);
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) c += __shfl_xor_sync(0xffffffffu, c, o);
  if (lane == 0) counts[b] = c;
}

// Exclusive scan of counts[0..n) into counts (in place) and counts[n] = total; one block.
__global__ void __launch_bounds__(1024) k_scan(int64_t* counts, int n) {
  __shared__ long long part[32];
  __shared__ long long carry;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  if (tid == 0) carry = 0;
  __syncthreads();
  for (int base = 0; base < n; base += 1024) {
    const int i = base + tid;
    const long long v = i < n ? counts[i] : 0;
    long long x = v;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const long long u = __shfl_up_sync(0xffffffffu, x, o);
      if (lane >= o) x += u;
    }
    if (lane == 31) part[warp] = x;
    __syncthreads();
    if (warp == 0) {
      long long y = part[lane];
#pragma unroll
      for (int o = 1; o < 32; o <<= 1) {
        const long long u = __shfl_up_sync(0xffffffffu, y, o);
        if (lane >= o) y += u;
      }
      part[lane] = y;
    }
    __syncthreads();
    const long long excl = carry + (warp ? part[warp - 1] : 0) + x - v;
    if (i < n) counts[i] = excl;
    __syncthreads();
    if (tid == 0) carry += part[31];
    __syncthreads();
  }
  if (tid == 0) counts[n] = carry;
}

// Writes the peaks of bin b at offsets[b] .. in ascending FFT order (one warp per bin).
__global__ void k_scatter(const uint32_t* __restrict__ bits, int n_bins, int n_words, int bin_lo,
                          const int64_t* __restrict__ offsets, uint32_t* __restrict__ out_fft,
                          uint32_t* __restrict__ out_bin, int64_t cap) {
  const int b = blockIdx.x * (blockDim.x / 32) + (threadIdx.x >> 5);
  const int lane = threadIdx.x & 31;
  if (b >= n_bins) return;
  int64_t pos0 = offsets[b];
  for (int w0 = 0; w0 < n_words; w0 += 32) {
    const int w = w0 + lane;
    uint32_t word = w < n_words ? bits[(int64_t)b * n_words + w] : 0u;
    const int c = __popc(word);
    int x = c;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const int u = __shfl_up_sync(0xffffffffu, x, o);
      if (lane >= o) x += u;
    }
    int64_t pos = pos0 + x - c;
    while (word) {
      const int bit = __ffs(word) - 1;
      word &= word - 1;
      if (pos < cap) {
        out_fft[pos] = (uint32_t)(w * 32 + bit);
        out_bin[pos] = (uint32_t)(bin_lo + b);
      }
      ++pos;
    }
    pos0 += __shfl_sync(0xffffffffu, x, 31);
  }
}

size_t align256(size_t v) { return (v + 255) / 256 * 256; }

// Equalise + select + compact from an input layout; `extra` bytes at the front of the scratch
// buffer are reserved for the caller (the FFT output).
// min(total, cap) to the caller's device word; a total above cap flags the context.
__global__ void k_finish_count(const int64_t* __restrict__ total, int64_t cap, int64_t* d_n,
                               unsigned int* flag) {
  if (threadIdx.x == 0) {
    const int64_t n = *total;
    if (n > cap) atomicOr(flag, GFH_FLAG_CAPACITY);
    *d_n = n < cap ? n : cap;
  }
}

// Equalise + select + compact from an input layout; `extra` bytes at the front of the scratch
// buffer are reserved for the caller (the FFT output).  With d_n the count goes to device memory
// and nothing synchronises; otherwise it is read back into *h_n.
template <class In>
int run_peaks(gfh_ctx* c, In in, int n_fft, int bin_lo, int bin_hi, double theta, uint32_t* d_fft,
              uint32_t* d_bin, int64_t cap, int64_t* h_n, size_t extra, int64_t* d_n = nullptr) {
  const int n_bins = bin_hi - bin_lo + 1;
  const int n_words = (n_fft + 31) / 32;
  const size_t o_bits = align256(extra);
  const size_t o_cnt = o_bits + align256((size_t)n_bins * n_words * 4);
  const size_t total = o_cnt + align256(((size_t)n_bins + 1) * 8);
  int rc = ensure_scratch(c, total);
  if (rc) return rc;
  char* base = (char*)c->pm_buf;
  uint32_t* bits = (uint32_t*)(base + o_bits);
  int64_t* cnt = (int64_t*)(base + o_cnt);
  cudaStream_t st = c->stream;
  GFH_CUDA_TRY(launch_equalise(in, n_fft, bin_lo, bin_hi, (float)theta, bits, n_words, st));
  k_count<<<(n_bins + 7) / 8, 256, 0, st>>>(bits, n_bins, n_words, cnt);
  GFH_CUDA_TRY(cudaGetLastError());
  k_scan<<<1, 1024, 0, st>>>(cnt, n_bins);
  GFH_CUDA_TRY(cudaGetLastError());
  k_scatter<<<(n_bins + 7) / 8, 256, 0, st>>>(bits, n_bins, n_words, bin_lo, cnt, d_fft, d_bin,
                                              cap);
  GFH_CUDA_TRY(cudaGetLastError());
  if (d_n) {
    k_finish_count<<<1, 32, 0, st>>>(cnt + n_bins, cap, d_n, c->d_flag);
    GFH_CUDA_TRY(cudaGetLastError());
    return GFH_OK;
  }
  GFH_CUDA_TRY(cudaMemcpyAsync(c->h_pinned, cnt + n_bins, 8, cudaMemcpyDeviceToHost, st));
  GFH_CUDA_TRY(cudaStreamSynchronize(st));
  *h_n = (int64_t)c->h_pinned[0];
  return *h_n > cap ? GFH_ERR_SIZE : GFH_OK;
}

bool band_ok(int n_fft, int bin_lo, int bin_hi) {
  return n_fft >= 1 && bin_lo - 1 - kWarm >= 1 && bin_hi >= bin_lo;
}

}  // namespace

// Equaliser, peak test and compaction on band spectra (bins j0 .. j0 + ld - 1 of each of n_fft
// rows); `extra` bytes at the front of the context scratch belong to the caller.
int gfh_band_peaks(gfh_ctx* c, const float2* d_x, int64_t ld, int32_t j0, int32_t n_fft,
                   int32_t bin_lo, int32_t bin_hi, double theta, uint32_t* d_fft_idx,
                   uint32_t* d_bin, int64_t cap, int64_t* h_n_peaks, size_t extra) {
  if (!band_ok(n_fft, bin_lo, bin_hi) || (int64_t)bin_lo - 1 - kWarm < j0 ||
      (int64_t)bin_hi + 1 > (int64_t)j0 + ld - 1)
    return GFH_ERR_ARG;
  return run_peaks(c, BandIn{d_x, ld, j0}, n_fft, bin_lo, bin_hi, theta, d_fft_idx, d_bin, cap,
                   h_n_peaks, extra);
}

size_t gfh_peaks_scratch(int32_t n_fft, int32_t bin_lo, int32_t bin_hi, size_t extra) {
  const int n_words = (n_fft + 31) / 32;
  return align256(extra) + align256((size_t)(bin_hi - bin_lo + 1) * n_words * 4) +
         align256(((size_t)(bin_hi - bin_lo + 2)) * 8);
}

// The context's scratch buffer, grown on demand (a growth waits for the stream first).
int ensure_scratch(gfh_ctx* c, size_t bytes) {
  if (c->pm_bytes >= bytes) return GFH_OK;
  if (c->pm_buf) {
    if (c->stream) cudaStreamSynchronize(c->stream);
    cudaFree(c->pm_buf);
    c->pm_buf = nullptr;
    c->pm_bytes = 0;
  }
  if (cudaMalloc(&c->pm_buf, bytes) != cudaSuccess) return GFH_ERR_NOMEM;
  c->pm_bytes = bytes;
  return GFH_OK;
}

int gfh_fft_plan(gfh_ctx* c, int N, int batch, bool c2c, cufftHandle* out) {
  gfh_ctx::FftPlan* slot = nullptr;
  for (auto& f : c->fft)
    if (f.valid && f.c2c == c2c && f.n == N && f.batch == batch) { slot = &f; break; }
  if (!slot) {
    slot = &c->fft[0];                       // a free slot, else the least recently used
    for (auto& f : c->fft) {
      if (!f.valid) { slot = &f; break; }
      if (f.used < slot->used) slot = &f;
    }
    if (slot->valid) {
      if (c->stream) cudaStreamSynchronize(c->stream);
      cufftDestroy(slot->h);
      slot->valid = false;
    }
    const int hop = N / 2;
    const int bins = c2c ? N : N / 2 + 1;
    int n[1] = {N};
    int inembed[1] = {N};
    int onembed[1] = {bins};
    if (cufftPlanMany(&slot->h, 1, n, inembed, 1, hop, onembed, 1, bins,
                      c2c ? CUFFT_C2C : CUFFT_R2C, batch) != CUFFT_SUCCESS)
      return GFH_ERR_CUDA;
    slot->valid = true;
    slot->c2c = c2c;
    slot->n = N;
    slot->batch = batch;
  }
  slot->used = ++c->fft_clock;
  if (cufftSetStream(slot->h, c->stream) != CUFFT_SUCCESS) return GFH_ERR_CUDA;
  *out = slot->h;
  return GFH_OK;
}

extern "C" int gfh_peaks_from_power(gfh_ctx* ctx, const float* d_power, int64_t ld, int32_t n_fft,
                                    int32_t bin_lo, int32_t bin_hi, double theta,
                                    uint32_t* d_fft_idx, uint32_t* d_bin, int64_t cap,
                                    int64_t* h_n_peaks) {
  if (!ctx || !d_power || !h_n_peaks || cap < 0 || (cap > 0 && (!d_fft_idx || !d_bin)) ||
      !band_ok(n_fft, bin_lo, bin_hi) || ld < (int64_t)bin_hi + 2)
    return GFH_ERR_ARG;
  GFH_CUDA_TRY(cudaSetDevice(ctx->device));
  return run_peaks(ctx, PowerIn{d_power, ld}, n_fft, bin_lo, bin_hi, theta, d_fft_idx, d_bin, cap,
                   h_n_peaks, 0);
}

namespace {

int peakmap_impl(gfh_ctx* ctx, const float* d_series, int64_t n_samples, double fs, double t_fft,
                 int32_t bin_lo, int32_t bin_hi, double theta, uint32_t* d_fft_idx,
                 uint32_t* d_bin, int64_t cap, int64_t* h_n_peaks, int64_t* d_n_peaks) {
  if (!ctx || !d_series || (!h_n_peaks && !d_n_peaks) || cap < 0 ||
      (cap > 0 && (!d_fft_idx || !d_bin)) || !(fs > 0.0) || !(t_fft > 0.0))
    return GFH_ERR_ARG;
  const double nd = fs * t_fft;
  if (!(nd >= 4.0) || nd > 1.0e8) return GFH_ERR_ARG;
  const int N = (int)(nd + 0.5);
  if (N % 2) return GFH_ERR_ARG;
  const int hop = N / 2;
  if (n_samples < N) return GFH_ERR_ARG;
  const int64_t nf64 = (n_samples - N) / hop + 1;
  if (nf64 > 0x7fffffff) return GFH_ERR_SIZE;
  const int n_fft = (int)nf64;
  const int nc = N / 2 + 1;
  if (!band_ok(n_fft, bin_lo, bin_hi) || bin_hi + 1 > N / 2) return GFH_ERR_ARG;
  GFH_CUDA_TRY(cudaSetDevice(ctx->device));
  cufftHandle plan;
  int rc0 = gfh_fft_plan(ctx, N, n_fft, false, &plan);
  if (rc0) return rc0;
  // Scratch layout: [complex spectra | peak bit matrix | bin counts]; sized once, up front.
  const size_t spec_bytes = (size_t)n_fft * nc * sizeof(float2);
  const int n_words = (n_fft + 31) / 32;
  const size_t need = align256(spec_bytes) +
                      align256((size_t)(bin_hi - bin_lo + 1) * n_words * 4) +
                      align256(((size_t)(bin_hi - bin_lo + 2)) * 8);
  int rc = ensure_scratch(ctx, need);
  if (rc) return rc;
  float2* spec = (float2*)ctx->pm_buf;
  if (cufftExecR2C(plan, const_cast<float*>(d_series), (cufftComplex*)spec) !=
      CUFFT_SUCCESS)
    return GFH_ERR_CUDA;
  return run_peaks(ctx, ComplexIn{spec, nc}, n_fft, bin_lo, bin_hi, theta, d_fft_idx, d_bin, cap,
                   h_n_peaks, spec_bytes, d_n_peaks);
}

}  // namespace

extern "C" int gfh_peakmap(gfh_ctx* ctx, const float* d_series, int64_t n_samples, double fs,
                           double t_fft, int32_t bin_lo, int32_t bin_hi, double theta,
                           uint32_t* d_fft_idx, uint32_t* d_bin, int64_t cap,
                           int64_t* h_n_peaks) {
  if (!h_n_peaks) return GFH_ERR_ARG;
  return peakmap_impl(ctx, d_series, n_samples, fs, t_fft, bin_lo, bin_hi, theta, d_fft_idx, d_bin,
                      cap, h_n_peaks, nullptr);
}

extern "C" int gfh_peakmap_async(gfh_ctx* ctx, const float* d_series, int64_t n_samples,
                                 double fs, double t_fft, int32_t bin_lo, int32_t bin_hi,
                                 double theta, uint32_t* d_fft_idx, uint32_t* d_bin, int64_t cap,
                                 int64_t* d_n_peaks) {
  if (!d_n_peaks) return GFH_ERR_ARG;
  return peakmap_impl(ctx, d_series, n_samples, fs, t_fft, bin_lo, bin_hi, theta, d_fft_idx, d_bin,
                      cap, nullptr, d_n_peaks);
}

// Peakmap of a complex series (the heterodyned series of the follow-up, Sec. V): complex-to-complex
// FFTs of the same interlaced boxcar frames, then the equaliser and peak test of the real path.
extern "C" int gfh_peakmap_complex(gfh_ctx* ctx, const float* d_z, int64_t n_samples, double fs,
                                   double t_fft, int32_t bin_lo, int32_t bin_hi, double theta,
                                   uint32_t* d_fft_idx, uint32_t* d_bin, int64_t cap,
                                   int64_t* h_n_peaks) {
  if (!ctx || !d_z || !h_n_peaks || cap < 0 || (cap > 0 && (!d_fft_idx || !d_bin)) ||
      !(fs > 0.0) || !(t_fft > 0.0))
    return GFH_ERR_ARG;
  const double nd = fs * t_fft;
  if (!(nd >= 4.0) || nd > 1.0e8) return GFH_ERR_ARG;
  const int N = (int)(nd + 0.5);
  if (N % 2) return GFH_ERR_ARG;
  const int hop = N / 2;
  if (n_samples < N) return GFH_ERR_ARG;
  const int64_t nf64 = (n_samples - N) / hop + 1;
  if (nf64 > 0x7fffffff) return GFH_ERR_SIZE;
  const int n_fft = (int)nf64;
  if (!band_ok(n_fft, bin_lo, bin_hi) || bin_hi + 1 > N - 1) return GFH_ERR_ARG;
  GFH_CUDA_TRY(cudaSetDevice(ctx->device));
  cufftHandle plan;
  int rc0 = gfh_fft_plan(ctx, N, n_fft, true, &plan);
  if (rc0) return rc0;
  const size_t spec_bytes = (size_t)n_fft * N * sizeof(float2);
  const int n_words = (n_fft + 31) / 32;
  const size_t need = align256(spec_bytes) +
                      align256((size_t)(bin_hi - bin_lo + 1) * n_words * 4) +
                      align256(((size_t)(bin_hi - bin_lo + 2)) * 8);
  int rc = ensure_scratch(ctx, need);
  if (rc) return rc;
  float2* spec = (float2*)ctx->pm_buf;
  if (cufftExecC2C(plan, (cufftComplex*)const_cast<float*>(d_z), (cufftComplex*)spec,
                   CUFFT_FORWARD) != CUFFT_SUCCESS)
    return GFH_ERR_CUDA;
  return run_peaks(ctx, ComplexIn{spec, N}, n_fft, bin_lo, bin_hi, theta, d_fft_idx, d_bin, cap,
                   h_n_peaks, spec_bytes);
}

// ---- statistical peakmaps (training and evaluation data of the tile proposer) -------------------

namespace {

// bits[(j - bin_lo) * n_words + w], bit l: FFT 32 w + l is a peak of the sample (one warp per word).
__global__ void k_synth_bits(uint64_t seed, uint64_t sample, int n_fft, int bin_lo, int n_bins,
                             int n_words, uint32_t p_noise24, uint32_t p_track24,
                             const int32_t* __restrict__ track, uint32_t* __restrict__ bits) {
  const int64_t q = (int64_t)blockIdx.x * (blockDim.x / 32) + (threadIdx.x >> 5);
  const int lane = threadIdx.x & 31;
  if (q >= (int64_t)n_bins * n_words) return;
  const int jl = (int)(q / n_words), w = (int)(q % n_words);
  const int i = w * 32 + lane;
  const bool pk = i < n_fft && gfh_synth_peak(seed, sample, (uint32_t)i, (uint32_t)(bin_lo + jl),
                                             p_noise24, track ? track[i] : -1, p_track24);
  const uint32_t word = __ballot_sync(0xffffffffu, pk);
  if (lane == 0) bits[q] = word;
}

}  // namespace

extern "C" int gfh_synth_peaks(gfh_ctx* ctx, uint64_t seed, int64_t sample, int32_t n_fft,
                               int32_t bin_lo, int32_t bin_hi, uint32_t p_noise24,
                               uint32_t p_track24, const int32_t* d_track, uint32_t* d_fft_idx,
                               uint32_t* d_bin, int64_t cap, int64_t* h_n_peaks) {
  if (!ctx || n_fft < 1 || bin_lo < 0 || bin_hi < bin_lo || !h_n_peaks || cap < 0 ||
      (cap > 0 && (!d_fft_idx || !d_bin)) || p_noise24 > (1u << 24) || p_track24 > (1u << 24))
    return GFH_ERR_ARG;
  GFH_CUDA_TRY(cudaSetDevice(ctx->device));
  const int n_bins = bin_hi - bin_lo + 1;
  const int n_words = (n_fft + 31) / 32;
  const size_t o_cnt = align256((size_t)n_bins * n_words * 4);
  int rc = ensure_scratch(ctx, o_cnt + align256(((size_t)n_bins + 1) * 8));
  if (rc) return rc;
  uint32_t* bits = (uint32_t*)ctx->pm_buf;
  int64_t* cnt = (int64_t*)((char*)ctx->pm_buf + o_cnt);
  cudaStream_t st = ctx->stream;
  const int64_t warps = (int64_t)n_bins * n_words;
  k_synth_bits<<<(unsigned)((warps + 7) / 8), 256, 0, st>>>(seed, (uint64_t)sample, n_fft, bin_lo,
                                                            n_bins, n_words, p_noise24, p_track24,
                                                            d_track, bits);
  GFH_CUDA_TRY(cudaGetLastError());
  k_count<<<(n_bins + 7) / 8, 256, 0, st>>>(bits, n_bins, n_words, cnt);
  k_scan<<<1, 1024, 0, st>>>(cnt, n_bins);
  k_scatter<<<(n_bins + 7) / 8, 256, 0, st>>>(bits, n_bins, n_words, bin_lo, cnt, d_fft_idx, d_bin, cap);
  GFH_CUDA_TRY(cudaGetLastError());
  GFH_CUDA_TRY(cudaMemcpyAsync(ctx->h_pinned, cnt + n_bins, 8, cudaMemcpyDeviceToHost, st));
  GFH_CUDA_TRY(cudaStreamSynchronize(st));
  *h_n_peaks = (int64_t)ctx->h_pinned[0];
  return *h_n_peaks > cap ? GFH_ERR_SIZE : GFH_OK;
}

// ---- allocation-free peak selection -------------------------------------------------------------
//
// For callers that cannot allocate device memory: a host application whose GPU memory is owned
// entirely by another allocator (a framework's caching pool, or a pipeline that reserves all
// device memory up front), where a library cudaMalloc could fail or where the implicit device
// synchronisation of cudaMalloc/cudaFree would stall the caller's other streams.  The scratch
// (peak bit matrix and per-bin counts) lives in this file-scope device array instead; every GPU
// that loads the library holds it until the process exits.

static __device__ __align__(256) unsigned char g_static_scratch[GFH_STATIC_SCRATCH_BYTES];

namespace {

constexpr int kMaxDevices = 64;
std::mutex g_static_mu;
void* g_static_addr[kMaxDevices] = {};

// Device address of g_static_scratch on the current device (looked up once per device: in host
// code the symbol's name is only a host-side stand-in, never a device address).
int static_scratch_addr(void** out) {
  int dev = -1;
  GFH_CUDA_TRY(cudaGetDevice(&dev));
  if (dev < 0 || dev >= kMaxDevices) return GFH_ERR_ARG;
  std::lock_guard<std::mutex> lock(g_static_mu);
  if (!g_static_addr[dev]) {
    void* p = nullptr;
    if (cudaGetSymbolAddress(&p, g_static_scratch) != cudaSuccess || !p) return GFH_ERR_CUDA;
    g_static_addr[dev] = p;
  }
  *out = g_static_addr[dev];
  return GFH_OK;
}

}  // namespace

extern "C" int gfh_peaks_from_power_static(void* stream, const float* d_power, int64_t ld,
                                           int32_t n_fft, int32_t bin_lo, int32_t bin_hi,
                                           double theta, uint32_t* d_fft_idx, uint32_t* d_bin,
                                           int64_t cap, int64_t* d_n_peaks) {
  if (!d_power || !d_n_peaks || cap < 0 || (cap > 0 && (!d_fft_idx || !d_bin)) ||
      !band_ok(n_fft, bin_lo, bin_hi) || ld < (int64_t)bin_hi + 2)
    return GFH_ERR_ARG;
  const int n_bins = bin_hi - bin_lo + 1;
  const int n_words = (n_fft + 31) / 32;
  const size_t o_cnt = align256((size_t)n_bins * n_words * 4);
  if (o_cnt + ((size_t)n_bins + 1) * 8 > GFH_STATIC_SCRATCH_BYTES) return GFH_ERR_SIZE;
  cudaStream_t st = (cudaStream_t)stream;
  if (st != nullptr && st != cudaStreamLegacy && st != cudaStreamPerThread) {
    // the array's address is the current device's: a created stream must belong to that device
    // (the default-stream handles always name the current device's)
    int cur = -1, sdev = -1;
    GFH_CUDA_TRY(cudaGetDevice(&cur));
    GFH_CUDA_TRY(cudaStreamGetDevice(st, &sdev));
    if (sdev != cur) return GFH_ERR_ARG;
  }
  void* base = nullptr;
  const int rc = static_scratch_addr(&base);
  if (rc) return rc;
  uint32_t* bits = (uint32_t*)base;
  int64_t* cnt = (int64_t*)((char*)base + o_cnt);
  // Every word of the bit matrix and every count is rewritten below, so nothing left by an
  // earlier call is read.
  GFH_CUDA_TRY(launch_equalise(PowerIn{d_power, ld}, n_fft, bin_lo, bin_hi, (float)theta, bits,
                               n_words, st));
  k_count<<<(n_bins + 7) / 8, 256, 0, st>>>(bits, n_bins, n_words, cnt);
  GFH_CUDA_TRY(cudaGetLastError());
  k_scan<<<1, 1024, 0, st>>>(cnt, n_bins);
  GFH_CUDA_TRY(cudaGetLastError());
  k_scatter<<<(n_bins + 7) / 8, 256, 0, st>>>(bits, n_bins, n_words, bin_lo, cnt, d_fft_idx,
                                              d_bin, cap);
  GFH_CUDA_TRY(cudaGetLastError());
  GFH_CUDA_TRY(cudaMemcpyAsync(d_n_peaks, cnt + n_bins, sizeof(int64_t), cudaMemcpyDeviceToDevice, st));
  return GFH_OK;
}
