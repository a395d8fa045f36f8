// Internal types shared by the translation units of libgfh (not part of the C ABI).
#pragma once

#include <cuda_runtime.h>
#include <cufft.h>
#include <cstdint>
#include <cstddef>
#include <vector>

#include "gfh.h"

#define GFH_FRAC_BITS 32

// Largest dynamic shared memory a block may use on sm_103a (227 KB).
constexpr size_t kMaxSmemBytes = 227 * 1024;
// dynamic shared memory a Hough tile may take: the kernels keep a few static bytes (tile counter)
constexpr size_t kHoughSmemLimit = kMaxSmemBytes - 64;

// Counter-based generator of the statistical peakmap model: the splitmix64 finaliser (Steele, Lea
// and Flood, "Fast splittable pseudorandom number generators", OOPSLA 2014) applied to a key built
// from (seed, sample, stream, FFT i, bin j); the top 24 bits are the cell's uniform.
__host__ __device__ __forceinline__ uint64_t gfh_mix64(uint64_t z) {
  z += 0x9E3779B97F4A7C15ull;
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
  return z ^ (z >> 31);
}

__host__ __device__ __forceinline__ uint32_t gfh_cell_u24(uint64_t seed, uint64_t sample,
                                                         uint32_t stream, uint32_t i, uint32_t j) {
  const uint64_t s = gfh_mix64(seed ^ (sample * 0xD1B54A32D192ED03ull) ^ ((uint64_t)stream << 56));
  return (uint32_t)(gfh_mix64(s ^ (((uint64_t)i << 32) | j)) >> 40);
}

// (FFT i, bin j) is a peak of the sample: a noise peak (stream 0 below p_noise24), or the cell of
// the injected track in FFT i and a track hit (stream 1 below p_track24).
__host__ __device__ __forceinline__ bool gfh_synth_peak(uint64_t seed, uint64_t sample, uint32_t i,
                                                       uint32_t j, uint32_t p_noise24,
                                                       int track_bin, uint32_t p_track24) {
  if (gfh_cell_u24(seed, sample, 0, i, j) < p_noise24) return true;
  return (int)j == track_bin && gfh_cell_u24(seed, sample, 1, i, j) < p_track24;
}

// Device-side error flag bits (gfh_check).
#define GFH_FLAG_UNSORTED 1u
#define GFH_FLAG_FFT_RANGE 2u
#define GFH_FLAG_CAPACITY 4u
#define GFH_FLAG_TIMEOUT 8u

#define GFH_CUDA_TRY(expr)                                \
  do {                                                    \
    cudaError_t e_ = (expr);                              \
    if (e_ != cudaSuccess) return GFH_ERR_CUDA;           \
  } while (0)

struct gfh_ctx {
  int device = 0;
  cudaStream_t stream = nullptr;
  int num_sms = 0;
  unsigned int* d_flag = nullptr;  // input-check flag
  // peakmap scratch (library-owned, grows on demand)
  void* pm_buf = nullptr;
  size_t pm_bytes = 0;
  // cuFFT plans of the interlaced frames (R2C for series, C2C for heterodyned series), kept for
  // the last few shapes so that searches alternating FFT lengths (Sec. VI.D portions) plan once
  struct FftPlan {
    cufftHandle h = 0;
    bool valid = false;
    bool c2c = false;
    int n = 0, batch = 0;
    unsigned long long used = 0;
  };
  static constexpr int kFftPlans = 4;
  FftPlan fft[kFftPlans];
  unsigned long long fft_clock = 0;
  // pinned host word for returning counts
  long long* h_pinned = nullptr;
  // bf16 bits of float(log(1 + c)) for c < kLogTable (image channel 0), built on the host
  uint16_t* d_log1p = nullptr;
};

constexpr int kLogTable = 4096;

// One map as the kernels see it.
struct MapDev {
  int32_t* out;             // [K][ld]
  const longlong2* UP;      // J: {U[j+1], U[j]} edge positions of bin j (upper f, lower f)
  const longlong2* BS;      // n_fft: {B_i, S_i}
  const int32_t* col_band;  // ld entries, -1 outside the analysis band / beyond n_x0
  const double* f0c;        // n_x0
  const double* f0n;        // n_x0
  int64_t* csr;             // J + 1 entries: first peak (absolute index) of bins bin_lo .. bin_hi+1
  unsigned long long* keys; // n_bands
  unsigned long long* sums; // 2: sum, sum of squares
  gfh_candidate* cands;     // n_bands (may be null)
  gfh_map_stats* stats;     // 1 (may be null)
  int64_t W;                // n_x0
  int64_t ld;               // ld_x0
  int64_t cells;            // analysis cells
  double x0_min, dx0, k_min, dk;
  int32_t K;
  int32_t bin_lo, bin_hi;
  int32_t n_fft;
  int32_t list;
  int32_t n_bands;
  int32_t csr_base;         // index of this map's first CSR entry in the plan-wide numbering
};

// Per map, for the coarse-tile search's FFT sub-ranges: an index of each bin's peaks by blocks of
// kFftBlock FFTs (built per execute, valid when the map's list holds each bin's peaks in FFT
// order) and the shift B_i + r S_i against i as a line through the table's first and last rows
// (the starting guess of a bin's FFT window, which the table then confirms).
constexpr int kFftBlock = 64;
struct CoarseMapDev {
  int32_t* fblk;            // [J][nb1]: offset in the bin's peaks of its first peak with FFT >= 64 b
  int32_t nb1;              // ceil(n_fft / 64) + 1 entries per bin
  int32_t list;             // the map's peak list
  int64_t b0, s0;           // B_0, S_0
  double db, ds;            // (B_last - B_0) / (n_fft - 1), (S_last - S_0) / (n_fft - 1)
};

// One tile of the accumulation kernel: k rows [row0, row0+nrows) x columns [col0, col0+ncols).
struct TileDev {
  int32_t map;
  int32_t row0;
  int32_t nrows;
  int32_t ncols;
  int64_t col0;
  int32_t bin_a;      // peaks with bins in [bin_a, bin_b] may touch the tile (bin_a > bin_b: none)
  int32_t bin_b;
  int32_t band_lo;    // candidate bands present in the tile's columns (band_hi < 0: none)
  int32_t band_hi;
  int32_t sub;        // coarse-tile search: walk only each bin's FFT sub-range (see hough_tile)
  int32_t reserved;
};

struct gfh_plan {
  gfh_ctx* ctx = nullptr;
  int n_maps = 0;
  std::vector<gfh_grid> grids;
  gfh_tile_config cfg{};
  void* d_buf = nullptr;       // tables, map descriptors, tiles
  size_t buf_bytes = 0;
  MapDev* d_maps = nullptr;
  TileDev* d_tiles = nullptr;          // tiles of x-direction maps follow the others
  int n_tiles = 0;                     // tiles differenced along k (rows > 0)
  int n_tiles_x = 0;                   // tiles of maps moving > 2 columns per k row: along x0
  std::vector<char> map_xd;            // per map: drawn in the x-direction form
  int max_tile_bands = 0;
  unsigned long long* d_keys = nullptr;  // all maps' keys and sums (zeroed per execute)
  size_t key_words = 0;
  int32_t csr_entries = 0;                // total CSR entries over maps
  int32_t* d_csr_map = nullptr;           // per CSR entry: map index
  bool select = false;
  int64_t* d_offsets_single = nullptr;    // scratch offsets for gfh_hough
  int* d_next = nullptr;                  // tile counters of the full search's two launches
  // the bound outputs, kept so that the autotuner can rebuild the plan with another tile shape
  std::vector<int32_t*> h_maps;
  std::vector<gfh_candidate*> h_cands;
  gfh_map_stats* d_stats = nullptr;
  // coarse tiles (gfh_plan_set_coarse): per (map, coarse tile) the fine tiles that cover it
  // (group coarse_k * coarse_x of a map = all of the map's tiles, for a full search)
  int coarse_k = 0, coarse_x = 0, max_sel = 0, max_fine = 0;
  void* d_coarse_buf = nullptr;
  TileDev* d_fine = nullptr;           // fine tiles, grouped by (map, coarse tile)
  int32_t* d_coarse_first = nullptr;   // n_maps * (coarse_k * coarse_x + 1) + 1 group offsets
  TileDev* d_sel_tiles = nullptr;      // the gathered tile list (worst case: every map in full)
  int* d_sel_count = nullptr;          // [0] list length, [1] next tile (persistent blocks)
  int sel_cap = 0;                     // capacity of d_sel_tiles
  CoarseMapDev* d_cmaps = nullptr;     // per map: FFT block index and shift line
  int* d_fft_unsorted = nullptr;       // per peak list: 1 if some bin's peaks are not in FFT order
  int n_list_flags = 0;                // entries of d_fft_unsorted (largest list index + 1)
  int sub_cap = 0;                     // bins per tile the sub-range walk holds in shared memory
  int fblk_entries = 0;                // largest J * nb1 over the maps (index build grid)
  int n_sub_tiles = 0;                 // coarse-group fine tiles flagged for the sub-range walk
};

// Host-side planning (gfh_host.cpp).
int gfh_host_tables(const gfh_grid* g, std::vector<int64_t>& U, std::vector<int64_t>& B,
                    std::vector<int64_t>& S);
int gfh_host_columns(const gfh_grid* g, std::vector<int32_t>& band, std::vector<double>& f0,
                     std::vector<double>& f0n);

// The context's scratch buffer (gfh_peakmap.cu), grown on demand.
int ensure_scratch(gfh_ctx* c, size_t bytes);
// Equaliser + peak test + compaction on band spectra d_x [n_fft][ld] holding bins j0 .. j0+ld-1
// (float2), with `extra` bytes at the front of the context scratch kept for the caller; the
// scratch that needs, to be ensured up front so that the caller's part is never reallocated.
int gfh_band_peaks(gfh_ctx* c, const float2* d_x, int64_t ld, int32_t j0, int32_t n_fft,
                   int32_t bin_lo, int32_t bin_hi, double theta, uint32_t* d_fft_idx,
                   uint32_t* d_bin, int64_t cap, int64_t* h_n_peaks, size_t extra);
size_t gfh_peaks_scratch(int32_t n_fft, int32_t bin_lo, int32_t bin_hi, size_t extra);
// A cuFFT plan of `batch` interlaced frames of N samples (hop N/2) on the context's stream.
int gfh_fft_plan(gfh_ctx* c, int N, int batch, bool c2c, cufftHandle* out);

// Launchers (gfh_hough.cu).
int gfh_launch_plan(gfh_plan* plan, const gfh_peaks* peaks);
int gfh_launch_plan_tiles(gfh_plan* plan, const gfh_peaks* peaks, const int32_t* d_coarse,
                          int n_sel, const int32_t* d_full);
int gfh_prepare_plan(gfh_plan* plan);   // one-time kernel attributes (outside any capture)
int gfh_launch_select(gfh_ctx* ctx, const int32_t* d_map, const MapDev& md, void* d_scratch);
