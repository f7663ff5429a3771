// Internal device-side layouts and kernel launchers of libmcao (not part of the C ABI).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

namespace mcao {

constexpr int kMaxEntries = 16;   // layers + DMs sampled along one direction
constexpr int kMaxNpx = 32;       // pupil samples per subaperture side
constexpr int kMaxNd = 32;        // detector pixels per subaperture side

// A phase grid sampled along a direction: a periodic turbulence layer or a bounded DM surface.
struct GridDev {
    const float* data;   // [n][n]
    int n;
    int periodic;        // 1: layer (wrap), 0: DM (clamp)
    double pixel;        // m
    double alt;          // m
    double vx, vy;       // m/s (0 for DMs)
    float sign;          // +1 layers, -1 DMs (residual = layers - DMs)
};

// One wavefront sensor.
struct WfsDev {
    int type;            // 0 NGS, 1 LGS
    int n_sub, n_px, n_fft, n_bin, n_det, N;  // N pupil samples across D
    int n_valid, slope0, frame0;              // frame0: first detector pixel in frame buffers
    int wfs_index;
    double dx;           // pupil sample pitch, m
    double theta_x, theta_y, height;
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
};

struct Ctx {
    const GridDev* grids;   // [n_grids]
    int n_grids;
    const WfsDev* wfs;      // [n_wfs]
    const StepState* st;
    double dt;
    unsigned long long seed;
    int noise;
};

// ---------------------------------------------------------------------------------------------
// launchers (return cudaGetLastError() of the launch)
// ---------------------------------------------------------------------------------------------

// One DM in the concatenated DM buffers.  T = C Gx^T restricted to the nonzero band of each
// Gaussian row, then S = Gy T (the Gaussian influence function factorises in x and y).
struct DmDesc {
    int nx, ny, surf_n, pad_;
    long long gx_off;    // Gx [surf_n][nx] in the table buffer
    long long gy_off;    // Gy [surf_n][ny]
    long long band_off;  // band_x [surf_n], band_y [surf_n] (lo, hi exclusive) in the band buffer
    long long map_off;   // act_map [ny][nx]: command index or -1
    long long tmp_off;   // T [ny][surf_n]
    long long surf_off;  // S [surf_n][surf_n]
};

struct DmLaunch {
    int n_dm;
    const DmDesc* desc;      // [n_dm] device
    const float* g;          // Gaussian tables
    const int2* band;        // bands
    const int* act_map;      // actuator maps
    const float* c;          // commands
    float* tmp;              // T buffers
    float* surf;             // surfaces
    long long tmp_total, surf_total;
    long long tmp_start[4], surf_start[4];   // per-DM prefix offsets (host copy, kernel args)
    StepState* st;           // begin of step: k = k_next (block 0)
};
constexpr int kMaxDms = 4;
cudaError_t launch_dm_surfaces(const DmLaunch& L, cudaStream_t s);

struct WfsLaunch {
    Ctx ctx;
    const SubapDev* subaps;  // [n_subaps] of the WFSs handled by this launch
    int n_subaps;
    const float* s_ref;
    float* slopes;
    float* lam_out;          // keep_frames: [total pixels] or null
    int* frame_out;
};

// variant = (n_px, n_fft, n_bin); returns cudaErrorInvalidValue when no kernel exists
bool wfs_variant_supported(int n_px, int n_fft, int n_bin, bool elongated);
cudaError_t wfs_prepare();   // kernel attributes (call once per device, outside stream capture)
cudaError_t launch_wfs(const WfsLaunch& L, int n_px, int n_fft, int n_bin, cudaStream_t s);

// residual phase of one WFS on its full pupil grid (tests)
cudaError_t launch_wfs_phase(const Ctx& ctx, int wfs, int N, float* out, cudaStream_t s);

struct ReconLaunch {
    const float* R;     // [rows_pad][ld]
    int n_cmd, n_slopes, ld, rows_pad;
    const float* s;     // [n_slopes]
    float* partial;     // [n_chunks][n_cmd]
    float* c;           // [n_cmd]
    float gain;
    StepState* st;      // k_next = k + 1 written by the reduce kernel (may be null)
};
constexpr int kReconRowBlock = 32;   // rows per block of the reconstructor product
constexpr int kReconChunk = 4096;    // slope columns per block
int recon_chunks(int n_slopes);
cudaError_t launch_recon(const ReconLaunch& L, cudaStream_t s);
cudaError_t launch_recon_reduce(const ReconLaunch& L, cudaStream_t s);

struct SciLaunch {
    Ctx ctx;
    int N, M;                 // pupil samples, FFT size
    double dx, theta_x, theta_y;
    float scale;              // lambda_ref / lambda_sci
    const float* amp;         // [N][N]
    float2* field;            // [N][N]
    float2* ft;               // [M][N] row-FFT output, transposed
    double* psf_t;            // [M][M] accumulated |FFT|^2, transposed, unshifted
    float2* sr_part;          // [n tiles] partial sums of the field
    int n_tiles;
    double sum_amp;
    int psf_every;
    const float2* w;          // [M] exp(-2 pi i k / M)
    int radices[8];
    int n_radices;
    StepState* st;
    SciAcc* acc;
};
cudaError_t sci_prepare(int M);   // kernel attributes (outside stream capture)
size_t sci_smem_bytes(int M);
cudaError_t launch_sci_field(const SciLaunch& L, cudaStream_t s);
cudaError_t launch_sci_rows(const SciLaunch& L, cudaStream_t s);
cudaError_t launch_sci_cols(const SciLaunch& L, cudaStream_t s);

cudaError_t launch_begin_step(StepState* st, cudaStream_t s);

}  // namespace mcao
