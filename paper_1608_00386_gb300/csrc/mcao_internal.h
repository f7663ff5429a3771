// Internal device-side layouts and kernel launchers of libmcao (not part of the C ABI).
#pragma once

#include <cuda_runtime.h>

#include <vector>
#include <stdint.h>

namespace mcao {

constexpr int kMaxEntries = 16;   // layers + DMs sampled along one direction

// Launch shapes of one simulation: the defaults, or what mcao_autotune measured fastest for its
// configuration (the knobs of the C ABI's MCAO_TUNE_* values, in that order).  None of them
// changes a result except tc_chunk, which regroups the tensor-core product's float32 sums.
struct Tuning {
    int sense_blocks_per_sm = 4;    // warp-per-subaperture sensing: grid cap, blocks per SM
    int recon_ctas_pct = 85;        // reconstructor slices: blocks per SM x 100
    int science_after_aux = 1;      // science waits for the block-per-subaperture sensors
    int tc_chunk = 8;               // tensor-core product: k-blocks per TMEM accumulator
    int multi_blocks_per_sm = 2;    // batched float32 product: blocks per SM
    int steps_per_graph = 1;        // steps captured in one graph launch (stage profiler off)
};
constexpr int kTuningKnobs = 6;
constexpr int kMaxNpx = 32;       // pupil samples per subaperture side
constexpr int kMaxNd = 32;        // detector pixels per subaperture side
constexpr int kMaxDms = 4;
constexpr int kMaxGridN = 65535;  // grid side (indices are packed in 16 bits)

// A phase grid (periodic turbulence layer or bounded DM surface) seen from one direction
// (a wavefront sensor or a science direction).  Grid coordinates are Q32.32 fixed point in
// grid samples: pupil sample (i, j) at step k sits at
//   x = ax + i bp + k vx,  y = ay + j bp + k vy,
// which is the cone-beam projection x_p (1 - h/H) + h theta plus the frozen-flow offset
// (k dt) v, converted to grid index units on the host in double precision.
struct GridView {
    const float* data;   // [n][n]
    int n;
    int periodic;        // 1: layer (wrap), 0: DM (index clamp into [0, n-1])
    long long ax, ay;    // grid index of pupil sample (0, 0) at step 0
    long long bp;        // grid samples per pupil sample
    long long vx, vy;    // grid samples per step (0 for DMs)
    float sign;          // +1 layers, -1 DMs (residual = layers - DMs)
    float inv_n;         // 1/n rounded to float (periodic wrap without a hardware divide)
};

// One wavefront sensor.
struct WfsDev {
    int type;            // 0 NGS, 1 LGS
    int n_sub, n_px, n_fft, n_bin, n_det, N;  // N pupil samples across D
    int n_valid, slope0, frame0;              // frame0: first detector pixel in frame buffers
    int rcol0;           // first column of this sensor's block in the padded slope / R layout
    int wfs_index;
    float scale;         // lambda_ref / lambda
    float n_photons, read_noise;
    const float* amp;    // [N][N] pupil amplitude
    float2 h[2 * kMaxNpx - 1];  // (-1)^u sum_{t<n_bin} exp(2 pi i u t / n_fft), u = -(n_px-1)..n_px-1
    float2 tw[kMaxNd];          // exp(2 pi i k / n_det)
};

// One valid subaperture.
struct SubapDev {
    int wfs;             // index into the WFS table
    int sx, sy;          // subaperture column / row
    int rank;            // rank among the WFS's valid subapertures
    float frac;          // illuminated fraction
    float elong_a;       // OTF(u) = exp(-elong_a (u . d)^2); 0 = no elongation
    float dir_x, dir_y;  // elongation direction
};

// Per-step device state: the DM kernel of a step copies k_next into k; the reconstructor
// reduction of the step writes k_next = k + 1.
struct StepState {
    long long k;         // step being computed
    long long k_next;    // completed steps
};

// Strehl / PSF accumulators of one science direction.
struct SciAcc {
    double sr_sum, sr_last;
    long long n_sr, n_psf;
    double var_sum, var_last;   // Marechal: residual phase variance (science band) per step
};

// Realizations: a simulation may advance n_real independent Monte-Carlo realizations of the
// same system together (own screens, DM commands, noise key seed + r, accumulators; shared
// geometry and reconstructor).  Per-realization arrays are realization-major with the strides
// below.
struct Ctx {
    const GridView* views;  // [n_real][n_views][n_grids]: WFSs first, then science directions
    long long view_stride;  // n_views * n_grids
    int n_grids;
    int n_real;
    const WfsDev* wfs;      // [n_wfs]
    const StepState* st;
    unsigned long long seed;   // realization r uses seed + r
    int noise;
};

// ---------------------------------------------------------------------------------------------
// DM surfaces
// ---------------------------------------------------------------------------------------------
// One DM in the concatenated DM buffers.  S = Gy C Gx^T (the Gaussian influence function
// factorises in x and y), evaluated per 64 x 64 block of the surface over the actuators whose
// weight on the block is at least 1e-10 (the bands are kept per 32-sample tile, the granularity
// the adjoint uses; a block takes the union of its two tiles' bands per axis).
struct DmDesc {
    int nx, ny, surf_n, tiles_x;   // tiles_x: 32-sample tiles per side of the surface
    long long gx_off;    // Gx [surf_n][nx] in the table buffer
    long long gy_off;    // Gy [surf_n][ny]
    long long gxt_off;   // Gx transposed, [nx][surf_n]
    long long gyt_off;   // Gy transposed, [ny][surf_n]
    long long tband_x;   // per 32-column tile: actuator columns [lo, hi) in the band buffer
    long long tband_y;   // per 32-row tile: actuator rows [lo, hi)
    long long map_off;   // act_map [ny][nx]: command index or -1
    long long surf_off;  // S [surf_n][surf_n]
    // misregistration: the DM's surface function evaluated at q = R(-rot)((x, y) - shift) / mag.
    // Without rotation it is folded into Gx and Gy; with rotation (general = 1) every sample
    // weighs the actuators within rc pitches of q directly (the tables are not used).
    int general;
    float cr, sr;        // cos, sin of the rotation
    float inv_mag, shx, shy;   // 1 / magnification; shift in m
    float dx, pitch;     // surface sample pitch, actuator pitch (m)
    float inv2s2;        // 1 / (2 sigma^2) of the influence function (DM coordinates)
    float rc;            // window radius in actuator pitches (weights below 1e-10 left out)
};
constexpr int kDmTile = 32;
constexpr int kDmMaxBand = 64;   // actuators per tile and axis (checked on the host)
constexpr int kDmBlock = 2 * kDmTile;   // surface samples per side of one block of the DM kernel
// shared memory of the DM kernel for blocks of at most nb actuators per axis
size_t dm_smem_bytes(int nb);
cudaError_t dm_prepare();   // kernel attribute admitting any block band <= 2 kDmMaxBand (outside capture)

struct DmLaunch {
    int n_dm;
    DmDesc desc[kMaxDms];    // by value: read from the parameter bank, no dependent load
    int nb;                  // largest actuator band of a block on either axis (shared memory)
    const float* g;          // Gaussian tables
    const int2* band;        // tile bands
    const int* act_map;      // actuator maps
    const float* c;          // commands
    float* surf;             // surfaces
    int tile_start[kMaxDms + 1];    // per-DM prefix of 64 x 64 surface blocks
    int n_real;              // realizations (grid y): commands c + r n_cmd, surfaces surf + r surf_stride
    int n_cmd;
    long long surf_stride;
    StepState* st;           // begin of step: k = k_next
    unsigned int* work;      // begin of step: the sensing kernels' work counters are zeroed
    int n_work;
};
cudaError_t launch_dm_surfaces(const DmLaunch& L, cudaStream_t s);
cudaError_t launch_begin_step(StepState* st, unsigned int* work, int n_work, cudaStream_t s);

// ---------------------------------------------------------------------------------------------
// wavefront sensors
// ---------------------------------------------------------------------------------------------
struct WfsLaunch {
    Ctx ctx;
    const SubapDev* subaps;  // [n_subaps] handled by this launch
    int n_subaps;
    const float* s_ref;
    float* slopes;
    float* slopes_pad;       // slopes again in the padded column layout of R (16-byte blocks)
    float* lam_out;          // keep_frames: [total pixels] or null
    int* frame_out;
    int slope_stride;        // per realization: slopes, padded slopes, frame pixels
    int pad_stride;
    long long frame_stride;
    // warp-per-subaperture route: with a work counter (zero at launch) the grid is capped at
    // max_blocks and warps take subapertures from the counter, so the launch adapts to the SM
    // slots that the concurrent reconstructor stream leaves; without one, one warp per subaperture
    unsigned int* work;
    int max_blocks;
};

bool wfs_variant_supported(int n_px, int n_fft, int n_bin, bool elongated);
bool wfs_variant_is_fft(int n_px, int n_fft, int n_bin);   // block-per-subaperture FFT route
cudaError_t wfs_prepare();   // kernel attributes (call once per device, outside stream capture)
cudaError_t launch_wfs(const WfsLaunch& L, int n_px, int n_fft, int n_bin, cudaStream_t s);

// residual phase of one WFS of realization r on its full pupil grid (tests)
cudaError_t launch_wfs_phase(const Ctx& ctx, int r, int wfs, int N, float* out, cudaStream_t s);

// ---------------------------------------------------------------------------------------------
// reconstructor
// ---------------------------------------------------------------------------------------------
constexpr int kReconRowBlock = 32;   // rows of R are padded to a multiple of this
constexpr int kReconChunk = 4096;    // maximum slope columns per chunk

// Element formats of the stored reconstructor (values of MCAO_DTYPE_*): float32; bfloat16;
// FP8 E4M3 with one float scale per row.  Elements are moved in 16-byte vectors of
// 16 / element-size elements.
constexpr int kReconF32 = 0, kReconBF16 = 1, kReconE4M3 = 2;
__host__ __device__ constexpr int recon_esize(int dtype) { return dtype == kReconF32 ? 4 : dtype == kReconBF16 ? 2 : 1; }

// One slice of the reconstructor product: the columns of one WFS's slope block (or of adjacent
// sensors sharing one kernel launch).
// R is held stage-tiled in HBM: for each slice, column chunk kc and row quad rq, a contiguous
// block of 4 x kc elements; inside it, stage t (128 vectors per row, fewer in the chunk's last
// stage; nv = the chunk's 16-byte vector count per row) holds its 4 row segments back to back,
// so every stage is one contiguous bulk copy of up to 8 KB.  The host picks the chunk width so
// that a chunk's last stage is not tiny (at least half a stage where it can).
struct ReduceLaunch {
    int n_cmd, n_chunks;
    const float* partial;   // [n_chunks][n_cmd], or null: the update is dc_in
    float* c;
    float gain;
    StepState* st;      // k_next = k + 1 (may be null)
    // second-order controller c_{k+1} = a1 c_k + a2 c_{k-1} + b0 dc_k + b1 dc_{k-1} (when set;
    // otherwise the pure integrator c += gain dc), over n_real realizations of n_cmd commands
    int use_ctl;
    float a1, a2, b0, b1;
    float* c_prev;
    float* dc_prev;
    const float* dc_in;  // [n_real][n_cmd] update (batched product), used when partial is null
    int n_real;
};
cudaError_t launch_recon_reduce(const ReduceLaunch& L, cudaStream_t s);

struct ReconLaunch {
    const unsigned char* R;   // stage-tiled reconstructor
    long long base;     // first byte of this slice in R
    int dtype;          // kReconF32 / kReconBF16 / kReconE4M3
    int n_cmd, n_rq;    // rows, row quads (rows padded to a multiple of 4)
    int col0;           // first column of the slice in the padded slope layout (multiple of 4)
    int len;            // columns in the slice
    int kc;             // columns per chunk (multiple of 16)
    int chunk0;         // first partial-sum slot of the slice
    const float* s;     // slopes in the padded layout (zeros in the padding, 16 spare floats)
    const float* scale; // per-row scales (kReconE4M3), else null
    float* partial;     // [n_chunks][n_cmd]
    int max_ctas;       // grid size cap (0: enough blocks for every item)
    unsigned int* work; // item counter, zero when the launch starts
    int* err;           // set to a nonzero code if a bounded wait gives up
};
constexpr int kReconRows = 4;        // rows per work item (row quad)
constexpr int kReconSeg = 128;       // 16-byte vectors per row and stage (at most)
constexpr int kSlopePadTail = 16;    // zero floats after the padded slopes (a vector may run past)
long long recon_slice_bytes(int n_rq, int len, int kc, int dtype);   // bytes of one slice in the tiled R
cudaError_t recon_prepare();   // kernel attributes (outside stream capture)
cudaError_t launch_recon(const ReconLaunch& L, cudaStream_t s);
// Per-row scales of the float32 R [rows][ld] (first cols columns) for kReconE4M3:
// max |R_r.| / 448 (1 for a zero row).
cudaError_t launch_recon_scales(const float* src, int rows, int cols, int ld, float* scale, cudaStream_t s);
// Re-lay the row-major, column-padded float32 R [rows][ld] (slice columns from col0) into the
// tiled slice, converting to the slice's element format.
cudaError_t launch_recon_tile(const float* src, int ld, const ReconLaunch& L, cudaStream_t s);
// Row-major codes [rows][cols] of R [rows][ld] in a reduced format (and its scales).
cudaError_t launch_quantize_rows(const float* src, int rows, int cols, int ld, int dtype, void* out,
                                 const float* scale, cudaStream_t s);
constexpr int kErrReconTimeout = 1;

// row-major float32 [rows][cols] -> [cols][ld_out] (float32, or bfloat16 codes when bf16 != 0);
// rows >= ld_out are not read, rows in [rows, ld_out) are written as zeros
cudaError_t launch_transpose(const float* src, int rows, int cols, void* out, int ld_out, int bf16, cudaStream_t st);

// ---------------------------------------------------------------------------------------------
// science
// ---------------------------------------------------------------------------------------------
struct SciLaunch {
    Ctx ctx;
    int view;                 // index of this direction's grid views
    int N, M;                 // pupil samples, FFT size
    float scale;              // lambda_ref / lambda_sci
    const float* amp;         // [N][N]
    float2* field;            // [N][N]
    float2* ft;               // [M][N] row-FFT output, transposed
    double* psf_t;            // [M][M] accumulated |FFT|^2, transposed, unshifted
    float4* sr_part;          // [n tiles] partial sums: field (re, im), A phi, A phi^2
    int n_tiles;
    double sum_amp;
    int psf_every;
    const float2* w;          // [M] exp(-2 pi i k / M)
    int radices[8];
    int n_radices;
    StepState* st;
    SciAcc* acc;
    // per realization r: field + r N^2, ft + r M N, psf_t + r M^2, sr_part + r n_tiles,
    // acc + r * acc_stride
    int acc_stride;
};
cudaError_t sci_prepare(int M);   // kernel attributes (outside stream capture)
size_t sci_smem_bytes(int M);
cudaError_t launch_sci_field(const SciLaunch& L, cudaStream_t s);
cudaError_t launch_sci_rows(const SciLaunch& L, cudaStream_t s);
cudaError_t launch_sci_cols(const SciLaunch& L, cudaStream_t s);

// ---------------------------------------------------------------------------------------------
// phase screens (von Karman, FFT method)
// ---------------------------------------------------------------------------------------------
size_t screen_fft_smem(int n);
cudaError_t launch_screen(int n, double pixel, double r0, double L0, unsigned long long seed, const int* radices,
                          int n_radices, float2* work, float2* W, float* out, cudaStream_t s);


// ---------------------------------------------------------------------------------------------
// adjoint of the noise-free sensing (interaction matrix, vector-Jacobian products)
// ---------------------------------------------------------------------------------------------
struct SensLaunch {
    Ctx ctx;
    int real;
    const SubapDev* subaps;  // one sensor's valid subapertures
    int n_subaps;
    float* sens;             // [n_slopes][P]: d slope / d phase on the slope's subaperture samples
    int P;                   // row length (largest n_px^2)
};
struct ProjLaunch {
    Ctx ctx;
    int real, n_layers, n_dms;
    const DmDesc* desc;
    const float* g;
    const int2* band;
    const int* act_map;
    const SubapDev* subaps;  // one sensor's valid subapertures
    int n_valid;
    const float* sens;
    int P;
    float* D;                // interaction matrix rows (or null)
    long long ld;
    const float* gvec;       // [n_vec][n_slopes] (or null)
    int n_vec, n_slopes;
    float* gc;               // [n_vec][n_cmd] accumulated (or null)
    int n_cmd;
    int* err;                // set when a footprint meets more actuators than a block holds
};
size_t sens_smem(int n_fft);
cudaError_t launch_sens(const SensLaunch& L, int n_fft, cudaStream_t s);
cudaError_t launch_dm_adjoint(const ProjLaunch& L, cudaStream_t s);
// Gauss-Newton records (16 doubles per slope row) of DM m's misregistration fit against D_meas
// (columns = DM m's commands, from cmd0), then their fixed-order sum
cudaError_t launch_misreg_gn(const ProjLaunch& L, int m, const float* D_meas, long long ld_meas, int cmd0, double* rec,
                             cudaStream_t s);
cudaError_t launch_misreg_sum(const double* rec, int n_rows, double* out, cudaStream_t s);
cudaError_t launch_phase_adjoint(const ProjLaunch& L, float* g_phase, long long phase_stride, long long phase_off,
                                 float* g_layers, long long layer_stride, const long long* layer_off, cudaStream_t s);

// per science direction: (long-exposure, instantaneous) Strehl ratio into out[2 q], out[2 q + 1]
cudaError_t launch_strehl_out(const SciAcc* acc, int n_sci, double* out, cudaStream_t s);
// one readout slot: ring_c[0..n_cmd) = c, ring_s[2q], ring_s[2q+1] = (long, last) Strehl of
// science direction q (n_cmd or n_sci may be 0)
cudaError_t launch_readout(const float* c, int n_cmd, const SciAcc* acc, int n_sci, float* ring_c, double* ring_s,
                           cudaStream_t s);

// twiddles of a science FFT of size M in the layout its kernels read (stage-major for the sizes
// with a compile-time transform, exp(-2 pi i m / M) otherwise)
std::vector<float2> sci_twiddles(int M);

// one bounded mbarrier wait that nothing satisfies: sets *err to kErrReconTimeout after about a
// second (self-check of the timeout path)
cudaError_t launch_wait_probe(int* err, cudaStream_t s);

// batched product for up to kMultiRhs realizations sharing R (column-major [K][rows_pad]):
// one pass over R, split-K partials, fixed-order reduction into out[r][i] = alpha D + beta out
constexpr int kMultiRhs = 16;
struct MultiLaunch {
    const void* R;           // float32 or bfloat16, column-major [K][rows_pad]
    int bf16;
    long long rows_pad;      // multiple of 4
    int n_cmd, K;
    float* s_t;              // [K][kMultiRhs] scratch (transposed slopes)
    float* partial;          // [multi_chunks(K)][kMultiRhs][n_cmd] scratch
};
int multi_chunks(int K);
cudaError_t multi_prepare();   // kernel attributes (outside stream capture)
cudaError_t launch_recon_multi(const MultiLaunch& L, int n_real, int pad_stride, const float* slopes_pad, float alpha,
                               float beta, float* out, int sm_count, int blocks_per_sm, cudaStream_t s);

// batched product for a bfloat16 R on the tensor cores (tcgen05, TMA, TMEM accumulators):
// out[r][i] = alpha sum_j R[i][j] s_r[j] + beta out[r][i] for every realization r, float32
// slopes (split exactly into three bfloat16 terms) and float32 accumulation; up to 64
// realizations per pass over R.  An FP8 E4M3 matrix (fp8 = 1) is stored as its code values
// (exact in bfloat16) with the per-row scales applied in the reduction: same product, the
// bytes of bfloat16.  tc_create converts the row-major float32 staging copy
// [rows_in][ld] (rows_in >= n_cmd) once and sizes the kernel for n_rhs realizations (outside
// stream capture); tc_launch queues the split, product and reduction kernels of every pass.
struct TcProduct;
cudaError_t tc_create(const float* R_rm, int rows_in, int ld, int n_cmd, int n_rhs, int sm_count, int fp8,
                      cudaStream_t st, TcProduct** out);
void tc_destroy(TcProduct* P);
cudaError_t tc_launch(TcProduct* P, const float* slopes_pad, int pad_stride, int n_real, float alpha, float beta,
                      float* out, int* err, int chunk, cudaStream_t st, int* launches);
long long tc_bytes(const TcProduct* P);   // bytes of its bfloat16 R

}  // namespace mcao
