/*
 * gfh.h - C ABI of the generalized FrequencyHough library for GB300 (sm_103a).
 *
 * The method (Miller et al., "A method to search for long duration gravitational wave transients
 * from isolated neutron stars using the generalized FrequencyHough", arXiv:1810.09784):
 *   Sec. III   a peakmap is the set of (time, frequency) points of equalised short-FFT spectra that
 *              exceed a threshold and are local maxima;
 *   Sec. IV    Eq. transform maps each peak frequency to x = f^(1-n); a power-law spin-down
 *              (Sec. II Eq. powlaws) is then the line x = x0 + (n-1) k (t - t0), so each peak is
 *              a line in the (x0, k) plane and the Hough map is the integer histogram of those
 *              lines; candidates are the highest counts per region, ranked by the critical ratio;
 *   Sec. VI.C  the x0 step is the finest one, dx0 = (n-1) df / f_max^n.
 * This library computes the peakmap, the integer Hough map and the per-band candidates on the GPU.
 *
 * Conventions for every entry point:
 *   - Device pointers ("d_" prefix) are allocated and owned by the caller; the library never frees
 *     them.  Host pointers ("h_" prefix or no prefix on plain structs) are read or written
 *     synchronously before the call returns.
 *   - All GPU work is issued on the stream bound to the context (gfh_create / gfh_set_stream) and
 *     is asynchronous unless a function says it synchronises.
 *   - Return value: GFH_OK (0) or a negative GFH_ERR_* code; nothing aborts and nothing throws.
 *     Data errors found on the device (unsorted peaks, out-of-range FFT index) are recorded in a
 *     device flag that gfh_check() reads and clears; the GPU context stays usable.
 *   - Peak lists are two parallel uint32 arrays: fft_idx (FFT number i, time t_i = t_first +
 *     i * t_hop from t0) and bin (frequency bin j, f_j = j * df), sorted by bin ascending (the
 *     order within one bin is free).  A peakmap never has two peaks in one (FFT, bin) cell.
 *   - A Hough map is int32 [n_k][ld_x0] row-major: row r is k_r = k_min + r dk, column m is the
 *     x0 interval [x0_min + m dx0, x0_min + (m+1) dx0).  Columns n_x0 .. ld_x0-1 are written 0.
 */
#ifndef GFH_H
#define GFH_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define GFH_OK 0
#define GFH_ERR_ARG (-1)      /* invalid argument: null pointer, n <= 1, empty band, bad size */
#define GFH_ERR_SIZE (-2)     /* capacity too small, or a size that overflows the index types */
#define GFH_ERR_CUDA (-3)     /* a CUDA runtime or cuFFT call failed */
#define GFH_ERR_INPUT (-4)    /* device-side input check failed (see gfh_check) */
#define GFH_ERR_TIMEOUT (-5)  /* a bounded device-side wait ran out */
#define GFH_ERR_NOMEM (-6)    /* a library-owned allocation failed */

typedef struct gfh_ctx gfh_ctx;
typedef struct gfh_plan gfh_plan;

/*
 * One Hough map (Sec. IV-VI).  The caller fills the request fields; gfh_grid_make fills the rest.
 *   n            braking index, n > 1 (Sec. I Eq. 1; Sec. II Eq. diff_powlaws fdot = -k f^n), or
 *                n = 0: the original FrequencyHough of Sec. III Eq. fdotslope (lines f0 = f - fdot t
 *                in the (f0, fdot) plane), mapped onto the same accumulator as x = -f, x0 = -f0,
 *                k = -fdot and x0 = x - k t (Eq. transform's x0 = x - (n-1) k t with (n-1) -> 1):
 *                dx0 = df, default dk = df / t_obs, candidates' x0 = -f0 and fdot0 = -k; only
 *                n = 0 accepts k_min < 0 (spin-up)
 *   df           frequency bin width 1/T_FFT [Hz]
 *   bin_lo..hi   peakmap band of this map, inclusive bins (f_j = j df); peaks outside are ignored
 *   n_fft        number of FFTs; t_first, t_hop give t_i = t_first + i t_hop from t0 [s]
 *   t_obs        observation time [s], used by the default k step
 *   n_k, k_min, dk   uniform k grid k_r = k_min + r dk; dk <= 0 selects dk = dx0/((n-1) t_obs),
 *                one x0 column of drift over t_obs per k row
 *   f_max        frequency of the finest x0 step (Sec. VI.C); <= 0 selects bin_hi * df
 *   ana_lo, ana_hi   analysis band [Hz): candidates are taken only in columns whose centre f0 lies
 *                inside it (Sec. IV: the peakmap band is wider than the analysed band)
 *   band_hz      candidate band width in f0 [Hz]: one candidate per band
 *   list         index of the peak list this map reads (gfh_plan_execute)
 * Derived: dx0 = (n-1) df / f_max^n; x0_min = x(f_top edge) - (n-1) max(k_max, 0) t_max - dx0;
 *   n_x0 = ceil((x(f_bottom edge) - (n-1) min(k_min, 0) t_max - x0_min)/dx0) + 1 (with 1 for
 *   n - 1 when n = 0); ld_x0 = n_x0 rounded up to 32;
 *   n_bands = ceil((ana_hi - ana_lo)/band_hz).
 */
typedef struct gfh_grid {
  double n;
  double df;
  int32_t bin_lo;
  int32_t bin_hi;
  int32_t n_fft;
  int32_t n_k;
  double t_first;
  double t_hop;
  double t_obs;
  double k_min;
  double dk;
  double f_max;
  double ana_lo;
  double ana_hi;
  double band_hz;
  int32_t list;
  int32_t n_bands;  /* derived */
  double dx0;       /* derived */
  double x0_min;    /* derived */
  int64_t n_x0;     /* derived */
  int64_t ld_x0;    /* derived */
} gfh_grid;

/*
 * One candidate (Sec. IV): the highest count of the map over all k rows and the columns of one f0
 * band, ties to the lowest row then the lowest column.  cr = (count - mu)/sigma with mu, sigma the
 * population mean and standard deviation over all analysis-band cells (0 when sigma = 0).
 * f0 = x0^(-1/(n-1)) (inverse of Eq. transform) and fdot0 = -k f0^n at the column centre.
 * count = -1 marks a band that holds no column.
 */
typedef struct gfh_candidate {
  int32_t band;
  int32_t row;
  int64_t col;
  int32_t count;
  int32_t reserved;
  double cr;
  double x0;
  double k;
  double f0;
  double fdot0;
} gfh_candidate;

/* Per-map statistics of the analysis-band cells: sum of counts, sum of squared counts, cells. */
typedef struct gfh_map_stats {
  int64_t sum;
  int64_t sum_sq;
  int64_t cells;
} gfh_map_stats;

/*
 * Peak lists for gfh_plan_execute: all lists concatenated in fft_idx / bin (device arrays);
 * list l is entries [offsets[l], offsets[l+1]) (device array of n_lists + 1 int64).
 */
typedef struct gfh_peaks {
  const uint32_t* fft_idx;
  const uint32_t* bin;
  const int64_t* offsets;
  int32_t n_lists;
} gfh_peaks;

/* Tile shape of the Hough kernel; zero fields pick the library default (16 x 3072, 512).  The
 * tile (rows x (cols + 2) int32 plus the candidate keys) must fit in 227 KB of shared memory.
 * form chooses how a warp draws its 32 peaks: 0 = each peak in its own form (interior peaks, clear
 * of the tile's edges on every row, in a shorter form than peaks near an edge; a warp holding both
 * runs both), 1 = one form per warp (the edge-following form for all 32 as soon as one needs it).
 * The maps are identical; 1 pays where many warps mix the two kinds of peak (narrow tiles, tall
 * maps).  The coarse-tile search always draws one form per warp. */
typedef struct gfh_tile_config {
  int32_t rows;     /* k rows per tile: 4, 8, 16 or 32 */
  int32_t cols;     /* x0 columns per tile: multiple of 128, at most 4096 */
  int32_t threads;  /* threads per block: 256 or 512, or 1024 with 16 or 32 rows */
  int32_t form;     /* drawing form: 0 or 1 */
} gfh_tile_config;

/* Context: binds a device and a stream (cudaStream_t passed as void*; NULL = legacy default). */
int gfh_create(gfh_ctx** out, int device, void* stream);
int gfh_destroy(gfh_ctx* ctx);
int gfh_set_stream(gfh_ctx* ctx, void* stream);
/* Synchronises the stream, then returns and clears the device-side check flag: GFH_OK,
 * GFH_ERR_TIMEOUT when a bounded device-side wait (tensor-core completion) ran out,
 * GFH_ERR_INPUT when the last calls saw unsorted peaks or an out-of-range index, or GFH_ERR_SIZE
 * when an asynchronous peakmap found more peaks than its capacity. */
int gfh_check(gfh_ctx* ctx);
const char* gfh_strerror(int code);

/* ---- host-side planning (no GPU needed) ---------------------------------------------------- */

/* Fills the derived fields of *g (Sec. VI.B-C).  Errors: GFH_ERR_ARG for an invalid request. */
int gfh_grid_make(gfh_grid* g);

/*
 * Fixed-point tables of one grid, for inspection (the plan builds its own copy).  Positions are in
 * x0 columns on a lattice of 2^-32 column, rounded down:
 *   h_U[e], e = 0..bin_hi-bin_lo+1: (x(f_e) - x0_min)/dx0 with f_e = (bin_lo + e - 1/2) df;
 *   h_B[i], h_S[i], i < n_fft: (n-1) k_min t_i / dx0 and (n-1) dk t_i / dx0.
 * A peak (i, j) covers, on row r, the half-open interval [h_U[j-bin_lo+1] - B_i - r S_i,
 * h_U[j-bin_lo] - B_i - r S_i) (Sec. IV: the line x0 = x - (n-1) k t_i of every x in the bin).
 * Any output pointer may be NULL.
 */
int gfh_grid_tables(const gfh_grid* g, int64_t* h_U, int64_t* h_B, int64_t* h_S);

/* Per column m < n_x0: candidate band (-1 outside the analysis band), f0 and f0^n of its centre. */
int gfh_grid_columns(const gfh_grid* g, int32_t* h_band, double* h_f0, double* h_f0n);

/*
 * Braking-index grid of Eq. dn_powlaws (Sec. VI.A): n_0 = n_lo, then n_{j+1} = n_j + dn_j with dn_j
 * the largest step (bisection to a relative 1e-9) for which the Eq. powlaws frequencies of n_j and
 * n_j + dn_j, at the same f0 and |fdot0| (k = |fdot0| / f0^n), differ by at most df over the
 * observation.  The difference is f0 |g(n2, u) - g(n1, u)| with g(n, u) = (1 + (n-1) u)^(-1/(n-1))
 * and u = |fdot0| t / f0; its maximum is taken over 64 f0 log-spaced in [f_min, f_max] and 256 equal
 * steps of u in [0, fdot_hi t_obs / f0].  The last point is n_hi.  Writes at most cap points to
 * h_n and their number to *n_out; GFH_ERR_SIZE when cap is too small (*n_out = points so far).
 */
int gfh_n_grid(double n_lo, double n_hi, double df, double f_min, double f_max, double fdot_hi,
               double t_obs, int32_t cap, double* h_n, int32_t* n_out);

/*
 * The k grid of Eq. dkeqn (Sec. VI.B) as uniform segments, each usable as the k grid of a
 * gfh_grid (k_min, dk, n_k): k runs from fdot_lo / f_max^n to the first row at or above
 * fdot_hi / f_min^n; the Eq. dkeqn step at k is |dk(k)| = k (1 - (1 + df/f_max)^(-n)) (the paper's
 * dk is negative; its size is used).  A segment starting at k_s has the step dk_s = |dk(k_s)| and
 * floor((growth - 1) / (1 - (1 + df/f_max)^(-n))) + 1 rows (at most max_rows), so no row is coarser
 * than growth times what the equation asks; the next segment starts one step after the last row.
 * growth = 1 gives one row per segment: the Eq. dkeqn grid itself.
 */
typedef struct gfh_k_segment {
  double k_min;
  double dk;
  int32_t n_k;
  int32_t reserved;
} gfh_k_segment;
int gfh_k_segments(double n, double df, double f_min, double f_max, double fdot_lo, double fdot_hi,
                   double growth, int32_t max_rows, int32_t cap, gfh_k_segment* h_out,
                   int32_t* n_out);

/*
 * Longer FFTs for later times (Sec. VI.D): the data from t0 to t_obs are split into portions
 * analysed with T_FFT = 2^L t_fft0, L = 0 .. max_levels-1.  With T_FFT a signal stays within one
 * frequency bin while |fdot| <= 1/T_FFT^2 (Eq. dot_tfft); once the spin-down has fallen by a factor
 * 4, T_FFT can double.  The spin-down is the largest any power law of braking index n with
 * f0 <= f_hi and |fdot0| <= fdot_hi can have at time t (Eq. powlaws): the fastest member's
 * fdot_hi (1 + (n-1) fdot_hi t / f_hi)^(-n/(n-1)) while t fdot_hi < f_hi, f_hi n^(-n/(n-1)) / t after
 * that (a slower member overtakes it).  Portion L spans [t_L, t_(L+1)) with t_L the first time that
 * bound falls to 1/T_L^2 (the last level runs to t_obs; times clipped to t_obs); levels whose span is
 * shorter than one T_FFT are left out, and data before the first portion (spin-down above
 * 1/t_fft0^2) is not analysed.  Every portion is searched with its own peakmap and maps on the common
 * t0 (grid t_first = portion start + T_FFT/2), so one signal has the same (x0, k) in all portions
 * and candidates of consecutive portions are compared with gfh_coincide (Sec. VI.D: coincidences
 * between the portions).  Host only.  GFH_ERR_SIZE when more than cap portions result.
 */
typedef struct gfh_portion {
  int32_t level;
  int32_t reserved;
  double t_begin;   /* [s from t0] */
  double t_end;
  double t_fft;
} gfh_portion;
int gfh_tfft_portions(double n, double f_hi, double fdot_hi, double t_fft0, double t_obs,
                      int32_t max_levels, int32_t cap, gfh_portion* h_out, int32_t* n_out);

/* ---- GPU entry points ----------------------------------------------------------------------- */

/*
 * Peak selection on given power spectra (Sec. III): d_power is float32 [n_fft][ld] row-major,
 * column j = bin j, ld >= bin_hi + 2.  Each spectrum is equalised by a clipped auto-regressive
 * mean S along frequency, in float32 with every operation IEEE-rounded (the paper fixes no
 * precision): S starts as the sum of the 128 bins below bin_lo - 1 times 2^-7 (so bin_lo >= 130);
 * then for bins bin_lo-1 .. bin_hi+1 in order: R_j = P_j / S, u = min(G P_j, 2.5 G S),
 * S = S + 2^-7 (u - S), with G = float32(1/(1 - e^-2.5)) = 1.08942544 and 2.5 G rounded to
 * 2.72356367.  Bin j in [bin_lo, bin_hi] is a peak iff R_j > theta and R_j > R_(j-1) and
 * R_j > R_(j+1) (theta rounded to float32; the paper uses 2.5, Sec. VII).
 * Output: at most cap peaks into d_fft_idx / d_bin, sorted by bin then FFT; *h_n_peaks = total
 * number of peaks found.  Synchronises the stream.  GFH_ERR_SIZE when the total exceeds cap
 * (the outputs then hold the first cap peaks of that order).
 */
int gfh_peaks_from_power(gfh_ctx* ctx, const float* d_power, int64_t ld, int32_t n_fft,
                         int32_t bin_lo, int32_t bin_hi, double theta, uint32_t* d_fft_idx,
                         uint32_t* d_bin, int64_t cap, int64_t* h_n_peaks);

/*
 * Peakmap of a time series (Sec. III): d_series float32 [n_samples] at fs Hz; FFTs of
 * N = round(fs t_fft) samples with hop N/2 (interlaced, boxcar window), FFT i starting at sample
 * i N/2, n_fft = (n_samples - N)/(N/2) + 1, bin_hi + 1 <= N/2; |X|^2 = re*re + im*im in float32
 * from a cuFFT R2C transform (unnormalised), then the equaliser and peak test of
 * gfh_peaks_from_power.  Same outputs, errors and synchronisation.
 */
int gfh_peakmap(gfh_ctx* ctx, const float* d_series, int64_t n_samples, double fs, double t_fft,
                int32_t bin_lo, int32_t bin_hi, double theta, uint32_t* d_fft_idx,
                uint32_t* d_bin, int64_t cap, int64_t* h_n_peaks);

/*
 * gfh_peakmap without any host synchronisation: the number of peaks written, min(total, cap), goes
 * to the device int64 *d_n_peaks (for example element 1 of a gfh_peaks offsets array whose element
 * 0 is 0), and a total above cap is reported by gfh_check as GFH_ERR_SIZE.  The first call with a
 * given (n_samples, fs, t_fft) builds the cuFFT plan and may grow the scratch: make it before any
 * stream capture; later calls only enqueue work and can be captured in a CUDA graph.
 */
int gfh_peakmap_async(gfh_ctx* ctx, const float* d_series, int64_t n_samples, double fs,
                      double t_fft, int32_t bin_lo, int32_t bin_hi, double theta,
                      uint32_t* d_fft_idx, uint32_t* d_bin, int64_t cap, int64_t* d_n_peaks);

/*
 * Plan for Hough maps plus candidates of n_maps grids (each made by gfh_grid_make), bound to
 * caller-owned outputs: h_maps[m] -> int32 [n_k][ld_x0] of grid m, h_cands[m] -> n_bands
 * gfh_candidate, d_stats -> n_maps gfh_map_stats (device).  h_cands or d_stats may be NULL (no
 * candidates).  The plan copies the grids, builds the fixed-point and column tables on the host
 * and uploads them; it owns that device memory until gfh_plan_destroy.  cfg may be NULL.
 * Errors: GFH_ERR_ARG, GFH_ERR_SIZE (n_k * n_x0 >= 2^32 - 1), GFH_ERR_NOMEM, GFH_ERR_CUDA.
 */
int gfh_plan_create(gfh_ctx* ctx, int32_t n_maps, const gfh_grid* grids, int32_t* const* h_maps,
                    gfh_candidate* const* h_cands, gfh_map_stats* d_stats,
                    const gfh_tile_config* cfg, gfh_plan** out);
int gfh_plan_destroy(gfh_plan* plan);

/*
 * Runs the plan on peak lists: every map reads list grids[m].list.  Writes all maps, and the
 * candidates and statistics if bound.  Asynchronous; no host synchronisation and no allocation,
 * so it can be captured in a CUDA graph.  Input errors are reported through gfh_check (a tile
 * whose bin range holds more than 2^31 - 2^20 peaks is not drawn: GFH_ERR_SIZE).
 */
int gfh_plan_execute(gfh_plan* plan, const gfh_peaks* peaks);

/*
 * Autotuner: times gfh_plan_execute on these peaks (reps runs each, CUDA events on the context's
 * stream) for the current tile shape and for every shape of rows {4, 8, 16} x cols {1024, 2048,
 * 3072, 4096} x threads {256, 512} (and 1024 threads for 16 rows) that fits in shared memory,
 * then the fastest shape with the other drawing form, and rebuilds the plan with the fastest.  The results are unchanged by the shape (the maps are
 * exact).  Synchronises; writes the bound outputs.  h_best / h_best_ms (may be NULL) receive the
 * chosen shape and its time.
 * The choice is cached for the life of the process, keyed by the plan's signature: the device
 * (compute capability, SM count), whether candidates are selected, and per map its k rows, x0
 * columns, bins, FFTs, line form and peak-density class (log2 of its list's peaks per (FFT, bin)
 * of its band, in quarter steps).  A plan whose signature is in the cache is rebuilt with the
 * cached shape and only that shape is timed.  Thread-safe.
 */
int gfh_plan_autotune(gfh_plan* plan, const gfh_peaks* peaks, int32_t reps,
                      gfh_tile_config* h_best, float* h_best_ms);

/* Number of plan signatures in the autotuner's cache, and emptying it (host only). */
int gfh_autotune_cache_size(void);
void gfh_autotune_cache_clear(void);

/* Convenience: one grid, one peak list of n_peaks entries; plan, execute, destroy. */
int gfh_hough(gfh_ctx* ctx, const uint32_t* d_fft_idx, const uint32_t* d_bin, int64_t n_peaks,
              const gfh_grid* g, int32_t* d_map, gfh_candidate* d_cands, gfh_map_stats* d_stats);

/*
 * Candidate selection alone on an existing map d_map [n_k][ld_x0] (Sec. IV), same rules and
 * outputs as the fused path of gfh_plan_execute.
 */
int gfh_select(gfh_ctx* ctx, const int32_t* d_map, const gfh_grid* g, gfh_candidate* d_cands,
               gfh_map_stats* d_stats);

/*
 * Candidates per "square" of an existing map d_map [n_k][ld_x0] (Sec. IV): the analysis-band
 * columns (contiguous: f0 falls with the column; GFH_ERR_ARG otherwise) are split into n_sx equal
 * chunks and the k rows into n_sk (chunk i of an axis of length L is [i L / n, (i + 1) L / n)).
 * Square q = j * n_sx + i (k chunk j, x0 chunk i) writes d_out[2 q] = its highest count (ties to the
 * lowest row, then column) and d_out[2 q + 1] = the highest count among its cells at least min_dk
 * rows from the first (Sec. IV: about 3 bins); band = q, reserved = 0 / 1; count = -1 where the
 * square has no cell (or no far row).  cr from the mean and deviation over all analysis cells,
 * which also go to d_stats (may be NULL).  n_k <= 65535.  Synchronous; its scratch is the
 * context's (shared with the peakmap builder, grown on demand).
 */
int gfh_select_squares(gfh_ctx* ctx, const int32_t* d_map, const gfh_grid* g, int32_t n_sx,
                       int32_t n_sk, int32_t min_dk, gfh_candidate* d_out, gfh_map_stats* d_stats);

/*
 * Coincidences (Sec. IV) between candidate sets a [na] and b [nb] (device, e.g. two detectors'
 * candidates on the same grid): for candidate i of a, d_match[i] = the index of the nearest
 * candidate of b by d = sqrt(((x0_b - x0_a)/dx0)^2 + ((k_b - k_a)/dk)^2) (ties to the lower
 * index) when d <= radius, else -1; d_dist[i] = that distance (-1 when a[i] or all of b have
 * count -1).  Records with count -1 take no part.  fp64, each operation IEEE-rounded.
 * Asynchronous.
 */
int gfh_coincide(gfh_ctx* ctx, const gfh_candidate* d_a, int32_t na, const gfh_candidate* d_b,
                 int32_t nb, double dx0, double dk, double radius, int32_t* d_match,
                 double* d_dist);

/* ---- follow-up of a candidate (Sec. V) ----------------------------------------------------------
 *
 * A candidate (f0, k, n) of the generalized search is followed up on the strain series: the series
 * is corrected by the candidate's spin-down phase (gfh_heterodyne), a peakmap with longer FFTs is
 * built from the corrected complex series (gfh_peakmap_complex), the original FrequencyHough (a grid
 * with n = 0) finds the residual (f0, fdot), and the peakmap corrected by that residual is projected
 * onto the frequency axis (gfh_project_peaks) for a new critical ratio.
 */

/*
 * Heterodyne correction (Sec. V Eq. phcor): d_out[s] = d_h[s] exp(-2 pi j c(t_s)) with t_s =
 * t_start + s / fs (seconds from t0 of Eq. powlaws) and c(t) = F(t) - f0 t, F the integral from t0
 * to t of f(t') = f0 / (1 + k (n-1) f0^(n-1) t')^(1/(n-1)):
 *   F = f0 (n-1) / ((n-2) a) ((1 + a t)^((n-2)/(n-1)) - 1), a = (n-1) k f0^(n-1)  (n != 2),
 *   F = (f0 / a) ln(1 + a t)                                                  (n = 2),
 * so that a power law of these parameters becomes a line at f0 (the sign makes the positive-
 * frequency half of a real signal monochromatic; the paper writes e^{j phi_sd} in its convention).
 *   d_h     float32 [n_samples] on the device (a 16-byte aligned pointer takes the vector path)
 *   d_out   complex64 [n_samples] as interleaved float32 pairs (re, im), caller-owned
 * Needs n > 1, k >= 0, t_start >= 0, f0 > 0.  Phase accuracy: c is exact in fp64 at anchors and
 * continued by its Taylor series to fourth order (the linear term exactly on a 2^-64 cycle lattice,
 * the others in float32); the anchor span is the longest power of two from 2^10 to 2^14 samples
 * over which the second..fourth-order terms stay below 1/8 cycle and the fifth-order term below
 * 1e-9 cycle at t_start (where the spin-down is fastest); GFH_ERR_ARG when even 2^10 samples is
 * too long.  The applied phase is the cycle fraction rounded to 2^-32 and then to float32.
 * Asynchronous; uses the context's scratch (one 32-byte anchor per span).
 */
int gfh_heterodyne(gfh_ctx* ctx, const float* d_h, int64_t n_samples, double fs, double t_start,
                   double f0, double k, double n, float* d_out);

/*
 * Peakmap of a complex series (Sec. III applied to the heterodyned series of Sec. V): d_z complex64
 * [n_samples] (interleaved re, im) at fs Hz; complex-to-complex FFTs (cuFFT, forward,
 * unnormalised) of the interlaced boxcar frames of gfh_peakmap (N = round(fs t_fft), hop N/2),
 * |X|^2 in float32, then the equaliser and peak test of gfh_peaks_from_power.  Bin j is frequency
 * j / t_fft for j < N/2; bin_hi + 1 <= N - 1.  Same outputs, errors and synchronisation as
 * gfh_peakmap.
 */
int gfh_peakmap_complex(gfh_ctx* ctx, const float* d_z, int64_t n_samples, double fs, double t_fft,
                        int32_t bin_lo, int32_t bin_hi, double theta, uint32_t* d_fft_idx,
                        uint32_t* d_bin, int64_t cap, int64_t* h_n_peaks);

/*
 * gfh_heterodyne followed by gfh_peakmap_complex in one pass that never forms the corrected series
 * or the full spectra (Sec. V Eq. phcor, Sec. III): only the bins the peak search reads, bin_lo - 129
 * .. bin_hi + 1, are computed for every frame, straight from the float32 series d_h.  Each frame's
 * bins j0 + k (j0 = bin_lo - 129, k < J, J = 256 or 512 as the band needs) are the first J outputs
 * of the frame's DFT after a rotation by j0 bins (added exactly to the phase lattice; it changes a
 * frame's spectrum by a constant phase, not its power): a decimated DFT of N = P J points (P / 32
 * groups of 32 residues, each a J-point radix-2 transform in shared memory, then a twiddled sum over
 * the residues).  Same arguments, outputs and synchronisation as the two calls, with
 * N = round(fs t_fft) a power of two >= 32 J (GFH_ERR_SIZE otherwise) and bin_hi + 1 <= N/2 - 1.
 * Accuracy: the heterodyne's (gfh_heterodyne), plus float32 transforms with sincospif twiddles
 * whose residue steps are 32-step recurrences; peak decisions then match the two-call path except
 * within rounding of a tie or of theta.  Uses the context's scratch (J bins x 8 bytes per frame).
 */
int gfh_heterodyne_band_peaks(gfh_ctx* ctx, const float* d_h, int64_t n_samples, double fs,
                              double t_start, double f0, double k, double n, double t_fft,
                              int32_t bin_lo, int32_t bin_hi, double theta, uint32_t* d_fft_idx,
                              uint32_t* d_bin, int64_t cap, int64_t* h_n_peaks);

/*
 * Projection of a bin-shifted peakmap onto frequency (Sec. V): peak (i, j) of the list (device
 * arrays of n_peaks) moves to bin j - floor(fdot t_i / df + 1/2), t_i = t_first + i t_hop (each
 * fp64 operation IEEE-rounded in that order), and d_counts[b - bin_lo] (int32, bin_hi - bin_lo + 1
 * <= 12288 entries, caller-owned) counts the peaks that land on bin b.  A line f0 + fdot t becomes
 * one column of the corrected peakmap.  Asynchronous.
 */
int gfh_project_peaks(gfh_ctx* ctx, const uint32_t* d_fft_idx, const uint32_t* d_bin,
                      int64_t n_peaks, double t_first, double t_hop, double df, double fdot,
                      int32_t bin_lo, int32_t bin_hi, int32_t* d_counts);

/* ---- statistical peakmaps and the learned tile proposer ------------------------------------------
 *
 * The paper proposes machine learning for future work (Sec. VIII); here a small convolutional
 * network ranks coarse (x0, k) tiles so that the exact Hough (above) can run on the best tiles only.
 * It never replaces the exact Hough: candidates always come from exact counts.
 *
 * Statistical peakmap model (training and evaluation data): cell (FFT i, bin j) of sample s is a
 * peak when u0(i, j) < p_noise24, or when j = track[i] and u1(i, j) < p_track24, where the 24-bit
 * uniforms u_stream(i, j) come from the splitmix64 finaliser mix(z) (Steele, Lea, Flood 2014):
 *   key = mix(seed ^ (s * 0xD1B54A32D192ED03) ^ (stream << 56)),  u = mix(key ^ (i << 32 | j)) >> 40.
 * p_*24 are probabilities times 2^24; track[i] is the bin of the injected power law in FFT i, or -1.
 */

/* Peak list (sorted by bin, then FFT) of sample `sample` for bins bin_lo..bin_hi; d_track has n_fft
 * entries or is NULL.  Synchronises; GFH_ERR_SIZE when the peaks exceed cap (count in *h_n_peaks). */
int gfh_synth_peaks(gfh_ctx* ctx, uint64_t seed, int64_t sample, int32_t n_fft, int32_t bin_lo,
                    int32_t bin_hi, uint32_t p_noise24, uint32_t p_track24, const int32_t* d_track,
                    uint32_t* d_fft_idx, uint32_t* d_bin, int64_t cap, int64_t* h_n_peaks);

/* Images of samples sample0 .. sample0 + batch - 1, bf16 [batch][256][256][2] (NHWC): pixel (tb, fb)
 * counts the peaks of FFTs [tb n_fft/256, (tb+1) n_fft/256) and bins bin_lo + [fb nb/256,
 * (fb+1) nb/256) (nb = bin_hi - bin_lo + 1 >= 256, n_fft >= 256); channel 0 = log(1 + count),
 * channel 1 = d_nplane[b].  d_tracks: [batch][n_fft]; d_p_track24: [batch]. */
int gfh_synth_images(gfh_ctx* ctx, uint64_t seed, int64_t sample0, int32_t batch, int32_t n_fft,
                     int32_t bin_lo, int32_t bin_hi, uint32_t p_noise24,
                     const uint32_t* d_p_track24, const int32_t* d_tracks, const float* d_nplane,
                     void* d_images);

/* The same images from peak lists: list l of `peaks` (each sorted by bin) into image l of d_images
 * [n_lists][256][256][2]; all maps share the band bin_lo..bin_hi and n_fft FFTs; d_nplane [n_lists].
 * Peaks outside the band are skipped; an FFT index >= n_fft sets the input flag (gfh_check).
 * GFH_ERR_ARG also for n_fft or nb of 2^24 or more.  Asynchronous. */
int gfh_peaks_to_images(gfh_ctx* ctx, const gfh_peaks* peaks, int32_t n_fft, int32_t bin_lo,
                        int32_t bin_hi, const float* d_nplane, void* d_images);

/*
 * The network (layer list in csrc/gfh_cnn.cu): input bf16 [B][256][256][2]; output 4097 logits per
 * image.  Class d * 64 + xt: a track starts (t = t0) in x0 tile xt (64 equal f0 ranges of the
 * analysis band, = 4 image columns when the image band is the analysis band) and drifts, over the
 * observation, between d K/64 and (d + 1) K/64 bins, K the map's k rows; a track on k row r
 * drifts r (f0 / f_max)^n bins (one x0 column per k row per t_obs with the default k step; one
 * column spans (f / f_max)^n bins, Eq. transform).  Class 4096 = no signal.
 * Parameters are one fp32 vector (gfh_cnn_param_count entries); the layout is fixed: for each 3x3
 * layer l = 1..5 its weights [cout][3][3][cin] then bias [cout]; the head [64][3][64] and bias [64];
 * the no-signal bias.  Weights start He-uniform from `seed`; AdamW (beta 0.9, 0.999, eps 1e-8).
 * All device memory (weights, optimiser state, activations for max_batch) is owned by the network.
 */
typedef struct gfh_cnn gfh_cnn;
int gfh_cnn_create(gfh_ctx* ctx, int32_t max_batch, uint64_t seed, gfh_cnn** out);
int gfh_cnn_destroy(gfh_cnn* net);
int64_t gfh_cnn_param_count(const gfh_cnn* net);
/* Host copies of the parameters and of the last gradients (either pointer may be NULL); sync. */
int gfh_cnn_get_params(gfh_cnn* net, float* h_params, float* h_grads);
/* Replace the parameters (and reset the optimiser state); sync. */
int gfh_cnn_set_params(gfh_cnn* net, const float* h_params);
/* Logits [batch][4097] fp32 into d_logits (may be NULL: kept inside). */
int gfh_cnn_forward(gfh_cnn* net, const void* d_images, int32_t batch, float* d_logits);
/* Gradients of the mean softmax cross-entropy for labels d_labels [batch] (int32 class); *h_loss =
 * mean loss (sync when h_loss is not NULL). */
int gfh_cnn_gradients(gfh_cnn* net, const void* d_images, const int32_t* d_labels, int32_t batch,
                      float* h_loss);
/* gfh_cnn_gradients followed by one AdamW step. */
int gfh_cnn_train_step(gfh_cnn* net, const void* d_images, const int32_t* d_labels, int32_t batch,
                       float lr, float weight_decay, float* h_loss);

/*
 * Training state for checkpoint and resume: the fp32 parameters, the AdamW first and second
 * moments (gfh_cnn_param_count entries each, host arrays) and the number of AdamW steps taken (the
 * bias corrections depend on it).  get: any pointer may be NULL; synchronises.  set: all three
 * arrays required; refreshes the bf16 weight copies; synchronises.  Resuming from a saved state
 * and taking the same batches gives bit-identical parameters to never having stopped.
 */
int gfh_cnn_get_state(gfh_cnn* net, float* h_params, float* h_m, float* h_v, int64_t* h_step);
int gfh_cnn_set_state(gfh_cnn* net, const float* h_params, const float* h_m, const float* h_v,
                      int64_t step);

/*
 * Copy of one internal tensor of the last forward (and backward) pass to the host, for checking
 * each stage on its own; synchronises.  which:
 *   GFH_CNN_ACT + l (l = 1..5)    activation after layer l, bf16 NHWC [batch][h][h][c]
 *                                 (h = 256, 128, 128, 64, 64; c = 32, 32, 64, 64, 64)
 *   GFH_CNN_DACT + l (l = 1..5)   gradient of the mean loss in layer l's pre-activation (the
 *                                 activation's gradient where the activation is > 0, else 0),
 *                                 bf16, same shape
 *   GFH_CNN_WBF16 + l (l = 0..4)  bf16 copy of the weights of layer l + 1, [cout][3][3][cin]
 *   GFH_CNN_POOLED                fp32 [batch][64 f][64 c], mean of activation 5 over its 64 rows
 *   GFH_CNN_LOGITS, GFH_CNN_DLOGITS   fp32 [batch][4097]: logits, d(mean loss)/d logits
 *   GFH_CNN_LOSS                  fp32 [batch] per-image cross-entropy
 * bytes = size of h_out; GFH_ERR_SIZE when it is too small, GFH_ERR_ARG for an unknown tensor or
 * a batch outside [1, max_batch].  Values past the last pass's batch are stale.
 */
#define GFH_CNN_ACT 0
#define GFH_CNN_DACT 10
#define GFH_CNN_WBF16 20
#define GFH_CNN_POOLED 30
#define GFH_CNN_LOGITS 31
#define GFH_CNN_DLOGITS 32
#define GFH_CNN_LOSS 33
int gfh_cnn_read_tensor(gfh_cnn* net, int32_t which, int32_t batch, void* h_out, int64_t bytes);

/*
 * Coarse-tile proposals from logits [batch][4097]: p = softmax(logits); class (d, xt) spreads p
 * evenly over k tiles kt in [floor(d gb), max(lo, ceil((d + 1) ga) - 1)] (both clamped to 63),
 * with d_gain [batch][64][2] = (ga, gb) = ((f_max / f_a)^n, (f_max / f_b)^n) for x0 tile xt over
 * [f_a, f_b).  Tiles kt * 64 + xt are ranked by score (descending, ties to the lower id; NaN
 * scores last); the first n leave resid_n = max(0, 1 - p(no signal) - their score sum), the
 * probability that the proposal misses a track.  tau >= 0: d_top [batch][k] keeps the first n
 * tiles for the smallest n <= k with resid_n <= tau (the rest -1); d_resid = resid_n; d_full (may
 * be NULL) = 1 where even resid_k > tau (the map needs the full search).  tau < 0: all k tiles,
 * resid_k, d_full = 0.  Asynchronous.
 */
int gfh_propose_tiles(gfh_ctx* ctx, const float* d_logits, int32_t batch, const float* d_gain,
                      int32_t k, float tau, int32_t* d_top, float* d_resid, int32_t* d_full);

/*
 * Non-learned proposer (the baseline the network is judged against): straight-line sums over
 * channel 0 of images d_images [batch][256][256][2] (as made by gfh_peaks_to_images for a band of
 * n_bins >= 256 bins equal to the analysis band, maps of n_k k rows).  Class (d, xt) is a track
 * starting in x0 tile xt (image columns 4 xt .. 4 xt + 3) that drifts (d + 1/2) n_k / 64 bins over
 * the observation: in time bin tb it lies off = floor(((2d + 1)(2tb + 1) n_k + 128 n_bins) /
 * (256 n_bins)) columns left of its start.  d_scores [batch][4096] (may be NULL) = the largest
 * over the four start columns of the sum over tb of the pixels on that line (pixels left of column
 * 0 add nothing); the sums are exact.  d_logits [batch][4097], ready for gfh_propose_tiles: with
 * z = (score - mean) / std over the image's scores (0 when they are all equal), class logit
 * beta z (beta >= 0) and no-signal logit LSE + det_c - det_a zmax, LSE = log sum exp(beta z) over
 * the classes and zmax the largest z, so that p(no signal) = 1 / (1 + exp(det_a zmax - det_c)).
 * Asynchronous.
 */
int gfh_line_scores(gfh_ctx* ctx, const void* d_images, int32_t batch, int32_t n_k, int32_t n_bins,
                    float beta, float det_a, float det_c, float* d_scores, float* d_logits);

/*
 * One 3x3 layer alone (tests): mode 0 forward out = relu(conv(in) + bias) into d_res (bf16 NHWC);
 * mode 1 input gradient into d_res (bf16) from d_dout masked by d_out > 0; mode 2 weight gradient
 * added into d_res (fp32 [cout][3][3][cin]) and bias gradient added into d_db.  (cin, cout, stride)
 * is one of (2, 32, 1) (the first layer: modes 0 and 2 only), (32, 32, 2), (32, 64, 1),
 * (64, 64, 2), (64, 64, 1); h = input height = width, a multiple of 16.
 */
int gfh_conv3x3(gfh_ctx* ctx, int32_t mode, int32_t cin, int32_t cout, int32_t stride,
                int32_t batch, int32_t h, const void* d_in, const void* d_w, const float* d_bias,
                const void* d_out, const void* d_dout, void* d_res, float* d_db);

/*
 * Exact Hough restricted to coarse tiles.  Each map of the plan is split into coarse_k x coarse_x
 * coarse tiles: k tile kt holds the rows r with floor(r coarse_k / K) = kt; x0 tile xt holds the
 * analysis columns whose centre f0 satisfies floor((f0 - ana_lo) / (ana_hi - ana_lo) * coarse_x) =
 * xt (clamped to [0, coarse_x - 1]); the coarse tile id is kt * coarse_x + xt.
 * gfh_plan_set_coarse (GFH_ERR_ARG for a plan with a map whose line moves more than two x0
 * columns per k row) builds, on the host, the plan's fine tiles (the plan's tile shape) that cover
 * every coarse tile, column ranges widened to multiples of 4; it must follow gfh_plan_create and may
 * be called again (an autotuned plan rebuilds them itself).  max_sel bounds n_sel below.
 * gfh_plan_execute_tiles computes the cells of the coarse tiles listed in d_coarse [n_maps][n_sel]
 * (device; ids outside [0, coarse_k coarse_x), e.g. -1, select nothing; an id listed twice for a
 * map is computed twice, and lists longer than the plan's tile capacity set the capacity flag
 * (gfh_check: GFH_ERR_SIZE) and are cut) exactly as gfh_plan_execute
 * does, and writes no other cell; a map with d_full[m] != 0 (d_full: device [n_maps], may be NULL)
 * is searched in full instead, exactly as by gfh_plan_execute.  All selected tiles of all maps run
 * in one launch of persistent blocks.  Candidates are the best computed cell of each band (count
 * -1 where no cell of the band was computed).  cr and the statistics come from sums over the
 * computed cells only (a cell computed twice counts twice) with the map's full cell count: they
 * are comparable with those of gfh_plan_execute only for maps searched in full.  A peak list whose
 * bins hold their peaks in FFT order (as gfh_peakmap emits them) lets narrow fine tiles read only
 * the peaks of the FFTs that can meet them; any other bin-sorted list is read in full, with the
 * same results.  Asynchronous, allocation-free, capturable.
 */
int gfh_plan_set_coarse(gfh_plan* plan, int32_t coarse_k, int32_t coarse_x, int32_t max_sel);
int gfh_plan_execute_tiles(gfh_plan* plan, const gfh_peaks* peaks, const int32_t* d_coarse,
                           int32_t n_sel, const int32_t* d_full);

/*
 * Failure-path check of the bounded device waits (the tensor-core kernels wait on mbarriers with a
 * limit of about a second): one block waits `cycles` SM cycles on an mbarrier that nothing arrives
 * at, then raises the timeout flag, so the next gfh_check returns GFH_ERR_TIMEOUT and clears it;
 * the context stays usable.  Asynchronous.  cycles <= 4e9.
 */
int gfh_wait_check(gfh_ctx* ctx, int64_t cycles);

/*
 * Measurement of the accumulator's roofline denominator: shared-memory atomicAdd throughput.
 * `blocks` blocks of `threads` threads each issue `iters` (a multiple of 4) 32-bit atomic adds of 1
 * to shared memory, cycling over four words per thread: mode 0 one word per bank per warp
 * (conflict-free), mode 1 one word per warp (all lanes the same address), mode 2 pseudo-random
 * words of a 32 KB array.  d_cycles [blocks] receives each block's elapsed SM cycles (clock64)
 * and d_sink [blocks] (zeroed by the caller) the sum of its array, blocks * threads * iters / blocks
 * per block.  The caller times the launch (CUDA events on the context's stream) for atomics per
 * second.  Asynchronous.  gfh_device_sms: the SM count of the context's device.
 */
int gfh_probe_smem_atomics(gfh_ctx* ctx, int32_t mode, int32_t blocks, int32_t threads,
                           int32_t iters, long long* d_cycles, int32_t* d_sink);
int gfh_device_sms(gfh_ctx* ctx, int32_t* h_sms);

/* ---- allocation-free entry point -------------------------------------------------------------
 *
 * The paper has no counterpart to this function: it is a service for callers that cannot
 * allocate device memory, e.g. an application whose GPU memory is entirely owned by another
 * allocator (a framework's caching pool, or a pipeline that reserves all device memory up front),
 * where a cudaMalloc inside the library could fail, and where the implicit device synchronisation
 * of cudaMalloc/cudaFree would stall the caller's other streams.
 *
 * Same peak selection as gfh_peaks_from_power (same inputs, same outputs, same order), but it needs
 * no context and allocates nothing (no cudaMalloc, no cudaFree, no allocating library routine).
 * Its scratch is one file-scope device array of GFH_STATIC_SCRATCH_BYTES (8 MiB), which every GPU
 * that loads the library holds until the process exits; it must hold the peak bit matrix and the
 * per-bin counts: 256-aligned (bins * ceil(n_fft/32) * 4) + (bins + 1) * 8 bytes, with bins =
 * bin_hi - bin_lo + 1 (for example 7800 bins x 5040 FFTs fits).  Larger requests return
 * GFH_ERR_SIZE and launch nothing.
 *   stream      cudaStream_t (as void*) of the current device (GFH_ERR_ARG for a stream of
 *               another device); all work is asynchronous on it
 *   d_n_peaks   device int64 that receives the total number of peaks, which may exceed cap; the
 *               outputs then hold the first cap peaks in (bin, FFT) order
 * The first call on a device looks up the array's device address (cudaGetSymbolAddress) with
 * that device current and keeps it for later calls.  A cudaDeviceReset of that device invalidates the kept address (the library must then
 * be reloaded).  All calls share the one array, so calls that overlap on the GPU (concurrent
 * streams, or several host threads) race and must be serialised by the caller; every call
 * rewrites all the scratch it reads, so no state carries over between calls.
 */
#define GFH_STATIC_SCRATCH_BYTES (8u << 20)
int gfh_peaks_from_power_static(void* stream, const float* d_power, int64_t ld, int32_t n_fft,
                                int32_t bin_lo, int32_t bin_hi, double theta,
                                uint32_t* d_fft_idx, uint32_t* d_bin, int64_t cap,
                                int64_t* d_n_peaks);

#ifdef __cplusplus
}
#endif

#endif /* GFH_H */
