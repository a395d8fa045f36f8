// Follow-up of a candidate (Sec. V) on sm_103a: the heterodyne correction of the strain series by
// the candidate's spin-down phase (Eq. phcor) and the projection of a bin-shifted peakmap onto the
// frequency axis.  (The longer-FFT peakmap of the corrected series is gfh_peakmap_complex; the
// original FrequencyHough on it is the accumulator with an n = 0 grid.)
//
// Heterodyne.  The residual phase c(t) = F(t) - f0 t (F the integral of Eq. powlaws) reaches 1e6-1e7
// cycles over a long observation, so it needs fp64 - and fp64 is the slow pipe of this GPU.  It is
// therefore evaluated in fp64 only at anchors every 2^10..2^14 samples (closed form, one thread per
// anchor), together with its first four derivatives.  Each sample then adds, modulo one cycle, the
// exact linear term on a 64-bit fixed-point lattice (integer multiply-add: no fp64) and the small
// quadratic..quartic terms in fp32; the fraction of a cycle, as an angle in [-pi, pi), feeds the
// hardware sine and cosine (absolute error 2^-21.4 there).  The kernel moves
// 4 bytes in and 8 bytes out per sample and is bound by HBM.
#include <algorithm>
#include <cmath>

#include "gfh_internal.h"

namespace {

// Anchor spans are powers of two from 2^10 to 2^14 samples, the longest the Taylor bounds allow.
constexpr int kMinSpanLog2 = 10, kMaxSpanLog2 = 14;

struct HetAnchor {
  unsigned long long C;   // c(t_a) mod 1 in units of 2^-64 cycles
  unsigned long long Q;   // (f(t_a) - f0) / fs mod 1: cycles per sample, 2^-64 units
  float e2, e3, e4;       // fdot/2, fddot/6, f'''/24 over fs^2, fs^3, fs^4: cycles per sample^k
  float pad;
};

struct HetParams {
  double fs, t_start, f0, k, n;
  double acoef;           // a = (n-1) k f0^(n-1) of Eq. powlaws: f = f0 (1 + a t)^(-1/(n-1))
  long long rot_bins;     // extra rotation by rot_bins / 2^rot_log2 cycles per sample (0: none)
  int rot_log2;
};

// x mod 1 on the 2^-64 lattice (x finite).
__device__ __forceinline__ unsigned long long frac64(double x) {
  double y = x - floor(x);
  if (!(y < 1.0)) y = 0.0;
  return __double2ull_rz(ldexp(y, 64));
}

// One thread per anchor: the residual phase and the derivatives of f at t_a = t_start + a span/fs.
__global__ void k_het_anchor(HetParams p, int64_t n_anchor, int span_log2,
                             HetAnchor* __restrict__ out) {
  const int64_t a = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (a >= n_anchor) return;
  const double t = p.t_start + (double)(a << span_log2) / p.fs;
  const double m1 = p.n - 1.0;
  const double acoef = p.acoef;
  double c = 0.0, d1 = 0.0, fd = 0.0, fdd = 0.0, fddd = 0.0;
  if (acoef != 0.0) {
    const double L = log1p(acoef * t);
    const double F = p.n == 2.0 ? (p.f0 / acoef) * L
                                : p.f0 * m1 / ((p.n - 2.0) * acoef) * expm1((p.n - 2.0) / m1 * L);
    c = F - p.f0 * t;
    const double f = p.f0 * exp(-L / m1);             // Eq. powlaws
    d1 = f - p.f0;
    const double g = acoef / (m1 * (1.0 + acoef * t));  // k f^(n-1): fdot = -g f (Eq. diff_powlaws)
    fd = -g * f;
    fdd = p.n * g * g * f;
    fddd = -p.n * (2.0 * p.n - 1.0) * g * g * g * f;
  }
  HetAnchor h;
  h.C = frac64(c);
  h.Q = frac64(d1 / p.fs);
  if (p.rot_bins != 0) {
    // + rot_bins s / 2^rot_log2 cycles at sample s = a span + m: exact on the 2^-64 lattice
    const unsigned long long nm = (1ull << p.rot_log2) - 1;
    const int sh = 64 - p.rot_log2;
    h.C += (((unsigned long long)p.rot_bins * ((unsigned long long)a << span_log2)) & nm) << sh;
    h.Q += ((unsigned long long)p.rot_bins & nm) << sh;
  }
  const double i1 = 1.0 / p.fs;
  h.e2 = (float)(0.5 * fd * i1 * i1);
  h.e3 = (float)(fdd / 6.0 * i1 * i1 * i1);
  h.e4 = (float)(fddd / 24.0 * i1 * i1 * i1 * i1);
  h.pad = 0.f;
  out[a] = h;
}

// z = h exp(-2 pi j c) for one sample m samples after its anchor.  The small terms (below 1/8
// cycle, host-checked) go onto the lattice through a 32-bit conversion (2^-34 cycle steps): a
// 64-bit float-to-integer conversion would run on the fp64 pipe.
__device__ __forceinline__ float2 het_sample(float h, const HetAnchor& A, int m) {
  const float mf = (float)m;
  const float small = mf * mf * (A.e2 + mf * (A.e3 + mf * A.e4));
  const int sf = __float2int_rn(small * 0x1p34f);
  const unsigned long long ph =
      A.C + (unsigned long long)m * A.Q + ((unsigned long long)(long long)sf << 30);
  const int top = (int)(ph >> 32);                                      // cycles in [-1/2, 1/2)
  float sn, cs;
  __sincosf((float)top * 0x1p-32f * 6.28318530717958647692f, &sn, &cs);   // |angle| <= pi
  return make_float2(h * cs, -h * sn);
}

// ---- band spectra of the heterodyned frames ------------------------------------------------------
//
// Frame f covers samples s0 = f hop .. s0 + N - 1 (N = 2^log2N, hop = N/2), and the follow-up needs
// its complex DFT only at bins j0 .. j0 + J - 1.  With y[s] = z[s] e^{-2 pi i j0 s / N} (z the
// heterodyned series; the rotation is folded into the anchors' phase and cycles per sample,
// exactly on the 2^-64 lattice, and changes each frame's spectrum by a constant phase only) the
// wanted outputs are the first J bins of the frame's DFT of y.  Writing n = P m + r (P = N / J): X[k] = sum_r W_N^(k r) Y_r[k] with Y_r the J-point DFT of
// y[s0 + P m + r] over m.  A block takes one frame: the residues in groups of 32 are staged as
// [m (bit-reversed)][r] (33-entry rows), transformed along m by radix-2 butterflies (each lane one
// residue), and thread k adds its output's share W_N^(k r) Y_r[k] (W_N^(k r0) by sincospif once per
// group, the 32 steps of W_N^k by recurrence).  No FFT of the whole frame is formed.
template <int J>
__global__ void __launch_bounds__(J, J == 256 ? 3 : 1) k_band_dft(const float* __restrict__ h,
                                                const HetAnchor* __restrict__ anchors,
                                                int span_log2, int log2N, int hop, int n_frames,
                                                int j0, float2* __restrict__ X) {
  constexpr int RG = 32, LD = RG + 1;
  constexpr int LOGJ = J == 256 ? 8 : 9;
  extern __shared__ float2 tile[];                   // [J][LD]
  __shared__ float2 tw[J / 2];                       // W_J^q = e^{-2 pi i q / J}
  const int tid = threadIdx.x;
  const int N = 1 << log2N, P = N >> LOGJ;
  const unsigned long long span_mask = (1ull << span_log2) - 1;
  for (int q = tid; q < J / 2; q += J) {
    float sn, cs;
    sincospif(-2.0f * (float)q / (float)J, &sn, &cs);
    tw[q] = make_float2(cs, sn);
  }
  // W_N^k for this thread's output k = tid
  float wks, wkc;
  sincospif(-2.0f * (float)tid / (float)N, &wks, &wkc);
  for (int f = blockIdx.x; f < n_frames; f += gridDim.x) {
    const int64_t s0 = (int64_t)f * hop;
    float2 acc = make_float2(0.f, 0.f);
    for (int r0 = 0; r0 < P; r0 += RG) {
      __syncthreads();                               // tile free (previous group consumed)
      // stage y[s0 + P m + r0 + rl] at row bitrev(m)
#pragma unroll 4
      for (int e = tid; e < J * RG; e += J) {
        const int m = e >> 5, rl = e & 31;
        const int64_t s = s0 + (int64_t)P * m + r0 + rl;
        const float2 y = het_sample(__ldg(h + s), anchors[s >> span_log2],
                                    (int)((unsigned long long)s & span_mask));
        const int mr = (int)(__brev((unsigned)m) >> (32 - LOGJ));
        tile[mr * LD + rl] = y;
      }
      __syncthreads();
      // radix-2 decimation in time along m, one residue per lane, two stages per pass: stages lg
      // and lg + 1 map the four entries base + {0, L, 2L, 3L} (L = 2^(lg-1)) onto themselves, so a
      // thread applies both stages' butterflies to them in registers (the same operations and
      // twiddles as stage by stage)
#pragma unroll
      for (int lg = 1; lg <= LOGJ; lg += 2) {
        const int L = 1 << (lg - 1);
        if (lg == 1) {
          // stages 1 and 2: every twiddle is 1 or -i, so the butterflies need no multiplies
#pragma unroll
          for (int it = 0; it < (J / 4) * RG / J; ++it) {
            const int e = tid + it * J;
            const int i0 = (e >> 5) << 2, rl = e & 31;
            const float2 a0 = tile[i0 * LD + rl], a1 = tile[(i0 + 1) * LD + rl];
            const float2 a2 = tile[(i0 + 2) * LD + rl], a3 = tile[(i0 + 3) * LD + rl];
            const float2 s0 = make_float2(a0.x + a1.x, a0.y + a1.y);
            const float2 d0 = make_float2(a0.x - a1.x, a0.y - a1.y);
            const float2 s1 = make_float2(a2.x + a3.x, a2.y + a3.y);
            const float2 d1 = make_float2(a2.x - a3.x, a2.y - a3.y);
            const float2 v = make_float2(d1.y, -d1.x);           // d1 times -i
            tile[i0 * LD + rl] = make_float2(s0.x + s1.x, s0.y + s1.y);
            tile[(i0 + 2) * LD + rl] = make_float2(s0.x - s1.x, s0.y - s1.y);
            tile[(i0 + 1) * LD + rl] = make_float2(d0.x + v.x, d0.y + v.y);
            tile[(i0 + 3) * LD + rl] = make_float2(d0.x - v.x, d0.y - v.y);
          }
        } else if (lg + 1 <= LOGJ) {
#pragma unroll
          for (int it = 0; it < (J / 4) * RG / J; ++it) {
            const int e = tid + it * J;
            const int b = e >> 5, rl = e & 31;
            const int grp = b >> (lg - 1), pp = b & (L - 1);
            const int i0 = (grp << (lg + 1)) + pp;
            float2 a0 = tile[i0 * LD + rl], a1 = tile[(i0 + L) * LD + rl];
            float2 a2 = tile[(i0 + 2 * L) * LD + rl], a3 = tile[(i0 + 3 * L) * LD + rl];
            const float2 w1 = tw[pp * (J >> lg)];
            const float2 w2 = tw[pp * (J >> (lg + 1))];
            const float2 w3 = tw[(pp + L) * (J >> (lg + 1))];
            float2 v = make_float2(a1.x * w1.x - a1.y * w1.y, a1.x * w1.y + a1.y * w1.x);
            a1 = make_float2(a0.x - v.x, a0.y - v.y);
            a0 = make_float2(a0.x + v.x, a0.y + v.y);
            v = make_float2(a3.x * w1.x - a3.y * w1.y, a3.x * w1.y + a3.y * w1.x);
            a3 = make_float2(a2.x - v.x, a2.y - v.y);
            a2 = make_float2(a2.x + v.x, a2.y + v.y);
            v = make_float2(a2.x * w2.x - a2.y * w2.y, a2.x * w2.y + a2.y * w2.x);
            tile[i0 * LD + rl] = make_float2(a0.x + v.x, a0.y + v.y);
            tile[(i0 + 2 * L) * LD + rl] = make_float2(a0.x - v.x, a0.y - v.y);
            v = make_float2(a3.x * w3.x - a3.y * w3.y, a3.x * w3.y + a3.y * w3.x);
            tile[(i0 + L) * LD + rl] = make_float2(a1.x + v.x, a1.y + v.y);
            tile[(i0 + 3 * L) * LD + rl] = make_float2(a1.x - v.x, a1.y - v.y);
          }
        } else {                                       // a last single stage (J = 512)
#pragma unroll
          for (int it = 0; it < (J / 2) * RG / J; ++it) {
            const int e = tid + it * J;
            const int b = e >> 5, rl = e & 31;
            const int grp = b >> (lg - 1), pos = b & (L - 1);
            const int i = (grp << lg) + pos, j = i + L;
            const float2 w = tw[pos * (J >> lg)];
            const float2 u = tile[i * LD + rl], v0 = tile[j * LD + rl];
            const float2 v = make_float2(v0.x * w.x - v0.y * w.y, v0.x * w.y + v0.y * w.x);
            tile[i * LD + rl] = make_float2(u.x + v.x, u.y + v.y);
            tile[j * LD + rl] = make_float2(u.x - v.x, u.y - v.y);
          }
        }
        __syncthreads();
      }
      // X[k] += sum_rl W_N^(k (r0 + rl)) Y_(r0 + rl)[k], k = tid
      float bs, bc;
      const int q0 = (int)(((long long)tid * r0) & (N - 1));
      sincospif(-2.0f * (float)q0 / (float)N, &bs, &bc);
      float2 wr = make_float2(bc, bs);               // W_N^(k r), r = r0 + rl
#pragma unroll 4
      for (int rl = 0; rl < RG; ++rl) {
        const float2 yv = tile[tid * LD + rl];
        acc.x += yv.x * wr.x - yv.y * wr.y;
        acc.y += yv.x * wr.y + yv.y * wr.x;
        wr = make_float2(wr.x * wkc - wr.y * wks, wr.x * wks + wr.y * wkc);
      }
    }
    X[(int64_t)f * J + tid] = acc;
  }
}

// Four samples per thread: float4 in, two float4 out (16-byte aligned buffers); a ragged tail is
// taken sample by sample.
__global__ void k_heterodyne(const float* __restrict__ h, int64_t n,
                             const HetAnchor* __restrict__ anchors, int span_log2,
                             float2* __restrict__ out, bool vec) {
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; q * 4 < n; q += stride) {
    const int64_t s0 = q * 4;
    const HetAnchor A = anchors[s0 >> span_log2];       // 4 samples never straddle an anchor
    const int m0 = (int)(s0 & ((int64_t(1) << span_log2) - 1));
    if (vec && s0 + 4 <= n) {
      const float4 v = __ldcs(reinterpret_cast<const float4*>(h + s0));
      const float2 z0 = het_sample(v.x, A, m0), z1 = het_sample(v.y, A, m0 + 1);
      const float2 z2 = het_sample(v.z, A, m0 + 2), z3 = het_sample(v.w, A, m0 + 3);
      float4* o = reinterpret_cast<float4*>(out + s0);
      __stcs(o, make_float4(z0.x, z0.y, z1.x, z1.y));
      __stcs(o + 1, make_float4(z2.x, z2.y, z3.x, z3.y));
    } else {
      for (int j = 0; j < 4 && s0 + j < n; ++j) out[s0 + j] = het_sample(h[s0 + j], A, m0 + j);
    }
  }
}

// Projection of bin-shifted peaks: one shared-memory histogram per block, then one global atomic
// per non-zero bin.  Every fp64 step is an explicitly rounded intrinsic (no contraction), so the
// shift equals the plain IEEE evaluation floor(fdot t_i / df + 1/2).
__global__ void k_project(const uint32_t* __restrict__ fft_idx, const uint32_t* __restrict__ bins,
                          int64_t n, double t_first, double t_hop, double df, double fdot,
                          int bin_lo, int n_bins, int32_t* __restrict__ counts) {
  extern __shared__ int hist[];
  for (int i = threadIdx.x; i < n_bins; i += blockDim.x) hist[i] = 0;
  __syncthreads();
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; p < n; p += stride) {
    const double t = __dadd_rn(t_first, __dmul_rn((double)fft_idx[p], t_hop));
    const double x = __dadd_rn(__ddiv_rn(__dmul_rn(fdot, t), df), 0.5);
    const long long j = (long long)bins[p] - (long long)floor(x) - bin_lo;
    if (j >= 0 && j < n_bins) atomicAdd(&hist[j], 1);
  }
  __syncthreads();
  for (int i = threadIdx.x; i < n_bins; i += blockDim.x)
    if (hist[i]) atomicAdd(&counts[i], hist[i]);
}

}  // namespace

extern "C" int gfh_heterodyne(gfh_ctx* ctx, const float* d_h, int64_t n_samples, double fs,
                              double t_start, double f0, double k, double n, float* d_out) {
  if (!ctx || n_samples < 0 || (n_samples > 0 && (!d_h || !d_out)) || !(fs > 0.0) ||
      !std::isfinite(fs) || !std::isfinite(t_start) || t_start < 0.0 || !(f0 > 0.0) ||
      !std::isfinite(f0) || !(k >= 0.0) || !std::isfinite(k) || !(n > 1.0) || !std::isfinite(n))
    return GFH_ERR_ARG;
  if (n_samples == 0) return GFH_OK;
  // |fdot| and its derivatives are largest at the start (f falls with t).  The anchor span is the
  // longest power of two (2^10 .. 2^14 samples) over which the quadratic..quartic terms stay below
  // 1/8 cycle and the first neglected (quintic) term below 1e-9 cycle; GFH_ERR_ARG when even 2^10
  // is too long.
  int span_log2 = -1;
  {
    const double m1 = n - 1.0;
    const double f = f0 / std::pow(1.0 + m1 * k * std::pow(f0, m1) * t_start, 1.0 / m1);
    const double g = k * std::pow(f, m1);
    for (int L = kMaxSpanLog2; L >= kMinSpanLog2 && span_log2 < 0; --L) {
      const double tau = std::ldexp(1.0, L) / fs;
      const double t2 = 0.5 * g * f * tau * tau;
      const double t3 = n * g * g * f / 6.0 * tau * tau * tau;
      const double t4 = n * (2.0 * n - 1.0) * g * g * g * f / 24.0 * tau * tau * tau * tau;
      const double t5 = n * (2.0 * n - 1.0) * (3.0 * n - 2.0) * g * g * g * g * f / 120.0 *
                        tau * tau * tau * tau * tau;
      if (t2 + t3 + t4 < 0.125 && t5 < 1e-9) span_log2 = L;
    }
  }
  if (span_log2 < 0) return GFH_ERR_ARG;
  GFH_CUDA_TRY(cudaSetDevice(ctx->device));
  const int64_t n_anchor = ((n_samples - 1) >> span_log2) + 1;
  int rc = ensure_scratch(ctx, (size_t)n_anchor * sizeof(HetAnchor));
  if (rc) return rc;
  HetAnchor* anchors = (HetAnchor*)ctx->pm_buf;
  cudaStream_t st = ctx->stream;
  const double acoef = (n - 1.0) * k * std::pow(f0, n - 1.0);
  k_het_anchor<<<(unsigned)((n_anchor + 127) / 128), 128, 0, st>>>(
      HetParams{fs, t_start, f0, k, n, acoef, 0, 0}, n_anchor, span_log2, anchors);
  GFH_CUDA_TRY(cudaGetLastError());
  const bool vec = ((uintptr_t)d_h % 16 == 0) && ((uintptr_t)d_out % 16 == 0);
  const int64_t quads = (n_samples + 3) / 4;
  int per_sm = 0;
  GFH_CUDA_TRY(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_heterodyne, 256, 0));
  const int64_t blocks = std::min<int64_t>((quads + 255) / 256,
                                           (int64_t)ctx->num_sms * (per_sm > 0 ? per_sm : 1));
  k_heterodyne<<<(unsigned)blocks, 256, 0, st>>>(d_h, n_samples, anchors, span_log2,
                                                 (float2*)d_out, vec);
  GFH_CUDA_TRY(cudaGetLastError());
  return GFH_OK;
}

extern "C" int gfh_project_peaks(gfh_ctx* ctx, const uint32_t* d_fft_idx, const uint32_t* d_bin,
                                 int64_t n_peaks, double t_first, double t_hop, double df,
                                 double fdot, int32_t bin_lo, int32_t bin_hi, int32_t* d_counts) {
  if (!ctx || n_peaks < 0 || (n_peaks > 0 && (!d_fft_idx || !d_bin)) || !d_counts ||
      bin_hi < bin_lo || !(df > 0.0) || !std::isfinite(t_first) || !std::isfinite(t_hop) ||
      !std::isfinite(fdot))
    return GFH_ERR_ARG;
  const int64_t nb = (int64_t)bin_hi - bin_lo + 1;
  if (nb > 12288) return GFH_ERR_SIZE;   // one shared-memory histogram per block (48 KB)
  GFH_CUDA_TRY(cudaSetDevice(ctx->device));
  cudaStream_t st = ctx->stream;
  GFH_CUDA_TRY(cudaMemsetAsync(d_counts, 0, (size_t)nb * sizeof(int32_t), st));
  if (n_peaks == 0) return GFH_OK;
  const int64_t blocks = std::min<int64_t>((n_peaks + 255) / 256, (int64_t)ctx->num_sms * 4);
  k_project<<<(unsigned)blocks, 256, (size_t)nb * sizeof(int), st>>>(
      d_fft_idx, d_bin, n_peaks, t_first, t_hop, df, fdot, bin_lo, (int)nb, d_counts);
  GFH_CUDA_TRY(cudaGetLastError());
  return GFH_OK;
}

extern "C" int gfh_heterodyne_band_peaks(gfh_ctx* ctx, const float* d_h, int64_t n_samples,
                                         double fs, double t_start, double f0, double k, double n,
                                         double t_fft, int32_t bin_lo, int32_t bin_hi, double theta,
                                         uint32_t* d_fft_idx, uint32_t* d_bin, int64_t cap,
                                         int64_t* h_n_peaks) {
  if (!ctx || !d_h || !h_n_peaks || cap < 0 || (cap > 0 && (!d_fft_idx || !d_bin)) ||
      !(fs > 0.0) || !(t_fft > 0.0) || !std::isfinite(t_start) || t_start < 0.0 ||
      !(f0 > 0.0) || !std::isfinite(f0) || !(k >= 0.0) || !std::isfinite(k) || !(n > 1.0) ||
      !std::isfinite(n))
    return GFH_ERR_ARG;
  const double nd = fs * t_fft;
  if (!(nd >= 1024.0) || nd > 1048576.0) return GFH_ERR_ARG;
  const int N = (int)(nd + 0.5);
  if ((N & (N - 1)) != 0) return GFH_ERR_ARG;            // a power of two
  int log2N = 0;
  while ((1 << log2N) < N) ++log2N;
  const int hop = N / 2;
  if (n_samples < N) return GFH_ERR_ARG;
  const int64_t nf64 = (n_samples - N) / hop + 1;
  if (nf64 > 0x7fffffff) return GFH_ERR_SIZE;
  const int n_fft = (int)nf64;
  // the equaliser reads bins bin_lo - 129 .. bin_hi + 1: J = 256 or 512 of them from j0
  const int j0 = bin_lo - 129;
  const int need = bin_hi + 1 - j0 + 1;
  if (j0 < 1 || bin_hi < bin_lo || bin_hi + 1 > N / 2 - 1) return GFH_ERR_ARG;
  const int J = need <= 256 ? 256 : 512;
  if (need > J || N < 32 * J) return GFH_ERR_SIZE;      // residues come in groups of 32
  int span_log2 = -1;
  {
    const double m1 = n - 1.0;
    const double f = f0 / std::pow(1.0 + m1 * k * std::pow(f0, m1) * t_start, 1.0 / m1);
    const double g = k * std::pow(f, m1);
    for (int L = kMaxSpanLog2; L >= kMinSpanLog2 && span_log2 < 0; --L) {
      const double tau = std::ldexp(1.0, L) / fs;
      const double t2 = 0.5 * g * f * tau * tau;
      const double t3 = n * g * g * f / 6.0 * tau * tau * tau;
      const double t4 = n * (2.0 * n - 1.0) * g * g * g * f / 24.0 * tau * tau * tau * tau;
      const double t5 = n * (2.0 * n - 1.0) * (3.0 * n - 2.0) * g * g * g * g * f / 120.0 *
                        tau * tau * tau * tau * tau;
      if (t2 + t3 + t4 < 0.125 && t5 < 1e-9) span_log2 = L;
    }
  }
  if (span_log2 < 0) return GFH_ERR_ARG;
  GFH_CUDA_TRY(cudaSetDevice(ctx->device));
  const int64_t n_anchor = ((n_samples - 1) >> span_log2) + 1;
  // scratch: [band spectra | anchors | the peak search's own]
  const size_t x_bytes = ((size_t)n_fft * J * sizeof(float2) + 255) / 256 * 256;
  const size_t a_bytes = ((size_t)n_anchor * sizeof(HetAnchor) + 255) / 256 * 256;
  int rc = ensure_scratch(ctx, gfh_peaks_scratch(n_fft, bin_lo, bin_hi, x_bytes + a_bytes));
  if (rc) return rc;
  float2* X = (float2*)ctx->pm_buf;
  HetAnchor* anchors = (HetAnchor*)((char*)ctx->pm_buf + x_bytes);
  cudaStream_t st = ctx->stream;
  const double acoef = (n - 1.0) * k * std::pow(f0, n - 1.0);
  k_het_anchor<<<(unsigned)((n_anchor + 127) / 128), 128, 0, st>>>(
      HetParams{fs, t_start, f0, k, n, acoef, (long long)j0, log2N}, n_anchor, span_log2, anchors);
  GFH_CUDA_TRY(cudaGetLastError());
  const size_t smem = (size_t)J * 33 * sizeof(float2);
  int per_sm = 0;
  if (J == 256) {
    GFH_CUDA_TRY(cudaFuncSetAttribute(k_band_dft<256>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    GFH_CUDA_TRY(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_band_dft<256>, 256, smem));
    const int grid = (int)std::min<int64_t>(n_fft, (int64_t)ctx->num_sms * std::max(per_sm, 1));
    k_band_dft<256><<<grid, 256, smem, st>>>(d_h, anchors, span_log2, log2N, hop, n_fft, j0, X);
  } else {
    GFH_CUDA_TRY(cudaFuncSetAttribute(k_band_dft<512>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    GFH_CUDA_TRY(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_band_dft<512>, 512, smem));
    const int grid = (int)std::min<int64_t>(n_fft, (int64_t)ctx->num_sms * std::max(per_sm, 1));
    k_band_dft<512><<<grid, 512, smem, st>>>(d_h, anchors, span_log2, log2N, hop, n_fft, j0, X);
  }
  GFH_CUDA_TRY(cudaGetLastError());
  return gfh_band_peaks(ctx, X, J, j0, n_fft, bin_lo, bin_hi, theta, d_fft_idx, d_bin, cap,
                        h_n_peaks, x_bytes + a_bytes);
}
