// Science path ("The Point Spread Functions (PSFs)" of arXiv:1608.00386: PSF at a user
// wavelength and pixel scale computed on the GPU; Strehl ratio from the PSF or the residual):
//   field E = A exp(i (lambda_ref / lambda) phi) along the science direction (source at
//   infinity), on-axis Strehl |sum E|^2 / (sum A)^2 every step, and every psf_every steps the
//   long-exposure PSF += |FFT2(E zero-padded to M x M)|^2 accumulated in double.
// The 2-D FFT runs as two passes of batched radix-4/5/2 Stockham FFTs in shared memory: rows of
// the field (zero-padded) written transposed, then rows of the transposed array; the PSF
// accumulator is therefore held transposed and unshifted, [kx][ky] (the host reorders it).
#include <algorithm>
#include <cmath>
#include <vector>

#include "device_common.cuh"
#include "mcao_internal.h"

namespace mcao {

namespace {

constexpr int kRowsPerBlock = 4;

// per-realization views of the launch (grid y = realization)
__device__ __forceinline__ SciLaunch sci_for_real(const SciLaunch& L0, int r) {
    SciLaunch L = L0;
    L.field += (long long)r * L.N * L.N;
    L.ft += (long long)r * L.M * L.N;
    L.psf_t += (long long)r * L.M * L.M;
    L.sr_part += (long long)r * L.n_tiles;
    L.acc += (long long)r * L.acc_stride;
    L.ctx.views += r * L.ctx.view_stride;
    return L;
}

__global__ void __launch_bounds__(256) sci_field_kernel(SciLaunch L0) {
    __shared__ AxisEnt s_ex[8][kMaxEntries * 8];
    __shared__ AxisEnt s_ey[8][kMaxEntries * 8];
    const SciLaunch L = sci_for_real(L0, blockIdx.y);
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int tiles_x = L.N / 8;
    const int tile = blockIdx.x * 8 + warp;
    if (tile >= tiles_x * tiles_x) return;
    const int i0 = (tile % tiles_x) * 8, j0 = (tile / tiles_x) * 8;
    const int n_grids = L.ctx.n_grids;
    const GridView* V = L.ctx.views + (long long)L.view * n_grids;
    tile_entries<8>(V, n_grids, L.ctx.st->k, i0, j0, s_ex[warp], s_ey[warp], lane, 32);
    __syncwarp();
    float sr = 0.0f, si = 0.0f, s1 = 0.0f, s2 = 0.0f;
    const int x = lane & 7;
#pragma unroll
    for (int hh = 0; hh < 2; ++hh) {
        const int y = (lane >> 3) + 4 * hh;
        float phi = tile_phase(V, n_grids, s_ex[warp], s_ey[warp], 8, x, y);
        float a = __ldg(L.amp + (long long)(j0 + y) * L.N + i0 + x);
        const float ph = L.scale * phi;
        float sn, cs;
        sincosf(ph, &sn, &cs);
        float2 e = make_float2(a * cs, a * sn);
        L.field[(long long)(j0 + y) * L.N + i0 + x] = e;
        sr += e.x;
        si += e.y;
        s1 = fmaf(a, ph, s1);
        s2 = fmaf(a * ph, ph, s2);
    }
    sr = warp_sum(sr);
    si = warp_sum(si);
    s1 = warp_sum(s1);
    s2 = warp_sum(s2);
    if (lane == 0) L.sr_part[tile] = make_float4(sr, si, s1, s2);
}

// Strehl of this step from the field partial sums, and the Marechal residual variance
// (piston removed, amplitude-weighted, science band) from the phase sums; fixed order, double
__device__ void finalize_strehl(const SciLaunch& L, double* red, int tid, int nthr) {
    double v[4] = {0.0, 0.0, 0.0, 0.0};
    // the thread's partials q = tid, tid + nthr, ... in that order, loaded eight at a time (the
    // loads of a batch in flight together)
    constexpr int kBatch = 8;
    for (int q0 = tid; q0 < L.n_tiles; q0 += kBatch * nthr) {
        float4 p[kBatch];
#pragma unroll
        for (int i = 0; i < kBatch; ++i) {
            const int q = q0 + i * nthr;
            p[i] = q < L.n_tiles ? L.sr_part[q] : make_float4(0.0f, 0.0f, 0.0f, 0.0f);
        }
#pragma unroll
        for (int i = 0; i < kBatch; ++i) {
            if (q0 + i * nthr >= L.n_tiles) break;
            v[0] += p[i].x;
            v[1] += p[i].y;
            v[2] += p[i].z;
            v[3] += p[i].w;
        }
    }
    for (int i = 0; i < 4; ++i) red[i * nthr + tid] = v[i];
    __syncthreads();
    for (int o = nthr / 2; o > 0; o >>= 1) {
        if (tid < o)
            for (int i = 0; i < 4; ++i) red[i * nthr + tid] += red[i * nthr + tid + o];
        __syncthreads();
    }
    if (tid == 0) {
        const double s = (red[0] * red[0] + red[nthr] * red[nthr]) / (L.sum_amp * L.sum_amp);
        L.acc->sr_sum += s;
        L.acc->sr_last = s;
        L.acc->n_sr += 1;
        const double mean = red[2 * nthr] / L.sum_amp;
        const double var = red[3 * nthr] / L.sum_amp - mean * mean;
        L.acc->var_sum += var;
        L.acc->var_last = var;
    }
    __syncthreads();
}

__device__ __forceinline__ bool psf_step(const SciLaunch& L) {
    return L.psf_every > 0 && (L.ctx.st->k % L.psf_every) == 0;
}

__global__ void __launch_bounds__(256) sci_rows_kernel(SciLaunch L0) {
    const SciLaunch L = sci_for_real(L0, blockIdx.y);
    extern __shared__ float4 smem_raw[];
    float2* A = reinterpret_cast<float2*>(smem_raw);
    float2* B = A + kRowsPerBlock * L.M;
    float2* W = B + kRowsPerBlock * L.M;
    double* red = reinterpret_cast<double*>(W + L.M);
    const int tid = threadIdx.x, nthr = blockDim.x;

    // the grid's last block only reduces the Strehl partials; it runs beside the FFT blocks
    if (blockIdx.x == gridDim.x - 1) {
        finalize_strehl(L, red, tid, nthr);
        return;
    }
    if (!psf_step(L)) return;

    const int row0 = blockIdx.x * kRowsPerBlock;
    for (int q = tid; q < L.M; q += nthr) W[q] = L.w[q];
    for (int q = tid; q < kRowsPerBlock * L.M; q += nthr) {
        int r = q / L.M, c = q - r * L.M;
        int row = row0 + r;
        A[q] = (row < L.N && c < L.N) ? L.field[(long long)row * L.N + c] : make_float2(0.0f, 0.0f);
    }
    __syncthreads();
    float2* R = stockham_fft(A, B, L.M, L.radices, L.n_radices, kRowsPerBlock, L.M, 1, W, tid, nthr);
    // transposed store: ft[c][row], four consecutive rows per column
    for (int q = tid; q < kRowsPerBlock * L.M; q += nthr) {
        int c = q / kRowsPerBlock, r = q - c * kRowsPerBlock;
        int row = row0 + r;
        if (row < L.N) L.ft[(long long)c * L.N + row] = R[r * L.M + c];
    }
}

__global__ void __launch_bounds__(256) sci_cols_kernel(SciLaunch L0) {
    const SciLaunch L = sci_for_real(L0, blockIdx.y);
    if (!psf_step(L)) return;
    extern __shared__ float4 smem_raw[];
    float2* A = reinterpret_cast<float2*>(smem_raw);
    float2* B = A + kRowsPerBlock * L.M;
    float2* W = B + kRowsPerBlock * L.M;
    const int tid = threadIdx.x, nthr = blockDim.x;
    const int c0 = blockIdx.x * kRowsPerBlock;
    for (int q = tid; q < L.M; q += nthr) W[q] = L.w[q];
    for (int q = tid; q < kRowsPerBlock * L.M; q += nthr) {
        int r = q / L.M, j = q - r * L.M;
        A[q] = (j < L.N) ? L.ft[(long long)(c0 + r) * L.N + j] : make_float2(0.0f, 0.0f);
    }
    __syncthreads();
    float2* R = stockham_fft(A, B, L.M, L.radices, L.n_radices, kRowsPerBlock, L.M, 1, W, tid, nthr);
    for (int q = tid; q < kRowsPerBlock * L.M; q += nthr) {
        int r = q / L.M, j = q - r * L.M;
        float2 v = R[q];
        float p = fmaf(v.x, v.x, v.y * v.y);   // frame intensity in float, accumulated in double
        L.psf_t[(long long)(c0 + r) * L.M + j] += (double)p;
    }
    if (blockIdx.x == 0 && tid == 0) L.acc->n_psf += 1;
}

// Compile-time-size versions of the two FFT passes (2 rows / columns per block, 256 threads);
// their twiddle table is stage-major (sci_twiddles).  Global loads are issued a whole pass at a
// time into registers before anything is stored, so that a block waits for about one memory
// round trip per pass rather than one per element.
constexpr int kCtRows = 2;
constexpr int kCtThreads = 256;

template <int M>
__global__ void __launch_bounds__(256) sci_rows_ct(SciLaunch L0) {
    const SciLaunch L = sci_for_real(L0, blockIdx.y);
    extern __shared__ float4 smem_raw[];
    float2* A = reinterpret_cast<float2*>(smem_raw);
    float2* B = A + kCtRows * M;
    float2* W = B + kCtRows * M;
    double* red = reinterpret_cast<double*>(W + M);
    const int tid = threadIdx.x, nthr = blockDim.x;
    // the grid's last block only reduces the Strehl partials (on the FP64 pipe of one SM, about
    // as long as an FFT block's work); it runs beside the FFT blocks
    if (blockIdx.x == gridDim.x - 1) {
        finalize_strehl(L, red, tid, nthr);
        return;
    }
    if (!psf_step(L)) return;
    static_assert((kCtRows * M) % kCtThreads == 0, "whole passes per thread");
    constexpr int PER = kCtRows * M / kCtThreads, PW = (M + kCtThreads - 1) / kCtThreads;
    const int row0 = blockIdx.x * kCtRows;
    {
        float2 w[PW], v[PER];
#pragma unroll
        for (int i = 0; i < PW; ++i) w[i] = tid + i * kCtThreads < M ? L.w[tid + i * kCtThreads] : make_float2(0.0f, 0.0f);
#pragma unroll
        for (int i = 0; i < PER; ++i) {
            const int q = tid + i * kCtThreads, r = q / M, c = q - r * M, row = row0 + r;
            v[i] = (row < L.N && c < L.N) ? L.field[(long long)row * L.N + c] : make_float2(0.0f, 0.0f);
        }
#pragma unroll
        for (int i = 0; i < PW; ++i)
            if (tid + i * kCtThreads < M) W[tid + i * kCtThreads] = w[i];
#pragma unroll
        for (int i = 0; i < PER; ++i) A[tid + i * kCtThreads] = v[i];
    }
    __syncthreads();
    float2* R = fft_tab<M>(A, B, kCtRows, W, tid, nthr);
#pragma unroll
    for (int i = 0; i < PER; ++i) {
        const int q = tid + i * kCtThreads, c = q / kCtRows, r = q - c * kCtRows, row = row0 + r;
        if (row < L.N) L.ft[(long long)c * L.N + row] = R[r * M + c];
    }
}

template <int M>
__global__ void __launch_bounds__(256) sci_cols_ct(SciLaunch L0) {
    const SciLaunch L = sci_for_real(L0, blockIdx.y);
    if (!psf_step(L)) return;
    extern __shared__ float4 smem_raw[];
    float2* A = reinterpret_cast<float2*>(smem_raw);
    float2* B = A + kCtRows * M;
    float2* W = B + kCtRows * M;
    const int tid = threadIdx.x, nthr = blockDim.x;
    static_assert((kCtRows * M) % kCtThreads == 0, "whole passes per thread");
    constexpr int PER = kCtRows * M / kCtThreads, PW = (M + kCtThreads - 1) / kCtThreads;
    const int c0 = blockIdx.x * kCtRows;
    {
        float2 w[PW], v[PER];
#pragma unroll
        for (int i = 0; i < PW; ++i) w[i] = tid + i * kCtThreads < M ? L.w[tid + i * kCtThreads] : make_float2(0.0f, 0.0f);
#pragma unroll
        for (int i = 0; i < PER; ++i) {
            const int q = tid + i * kCtThreads, r = q / M, j = q - r * M;
            v[i] = (j < L.N) ? L.ft[(long long)(c0 + r) * L.N + j] : make_float2(0.0f, 0.0f);
        }
#pragma unroll
        for (int i = 0; i < PW; ++i)
            if (tid + i * kCtThreads < M) W[tid + i * kCtThreads] = w[i];
#pragma unroll
        for (int i = 0; i < PER; ++i) A[tid + i * kCtThreads] = v[i];
    }
    // this block's PSF accumulator entries, read while the transform runs
    double acc[PER];
    double* psf = L.psf_t + (long long)c0 * M;
#pragma unroll
    for (int i = 0; i < PER; ++i) acc[i] = psf[tid + i * kCtThreads];
    __syncthreads();
    float2* R = fft_tab<M>(A, B, kCtRows, W, tid, nthr);
#pragma unroll
    for (int i = 0; i < PER; ++i) {
        const int q = tid + i * kCtThreads;
        const float2 v = R[q];
        const float p = fmaf(v.x, v.x, v.y * v.y);   // frame intensity in float, accumulated in double
        psf[q] = acc[i] + (double)p;
    }
    if (blockIdx.x == 0 && tid == 0) L.acc->n_psf += 1;
}

template <int M>
size_t ct_smem() {
    return sizeof(float2) * (2 * kCtRows * (size_t)M + M) + sizeof(double) * 4 * 256;
}

template <int M>
cudaError_t ct_prepare() {
    cudaError_t e = cudaFuncSetAttribute((const void*)sci_rows_ct<M>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)ct_smem<M>());
    if (e != cudaSuccess) return e;
    return cudaFuncSetAttribute((const void*)sci_cols_ct<M>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                (int)ct_smem<M>());
}

template <int M>
cudaError_t ct_rows(const SciLaunch& L, cudaStream_t s) {
    sci_rows_ct<M><<<dim3((unsigned)((L.N + kCtRows - 1) / kCtRows + 1), (unsigned)L.ctx.n_real), 256, ct_smem<M>(), s>>>(L);
    return cudaGetLastError();
}

template <int M>
cudaError_t ct_cols(const SciLaunch& L, cudaStream_t s) {
    sci_cols_ct<M><<<dim3((unsigned)(M / kCtRows), (unsigned)L.ctx.n_real), 256, ct_smem<M>(), s>>>(L);
    return cudaGetLastError();
}

// sizes with a compile-time kernel; other sizes use the generic one
#define MCAO_SCI_CT_SIZES(X) X(128) X(256) X(512) X(640) X(1024) X(1280) X(2048)

size_t fft_smem_bytes(int M) {
    return sizeof(float2) * (2 * kRowsPerBlock * (size_t)M + M) + sizeof(double) * 4 * 256;
}

cudaError_t set_smem(const void* fn, size_t bytes) {
    return cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
}

}  // namespace

cudaError_t launch_sci_field(const SciLaunch& L, cudaStream_t s) {
    int tiles = (L.N / 8) * (L.N / 8);
    sci_field_kernel<<<dim3((unsigned)((tiles + 7) / 8), (unsigned)L.ctx.n_real), 256, 0, s>>>(L);
    return cudaGetLastError();
}

bool sci_ct_size(int M) {
#define MCAO_CT_IS(n) \
    if (M == n) return true;
    MCAO_SCI_CT_SIZES(MCAO_CT_IS)
#undef MCAO_CT_IS
    return false;
}

std::vector<float2> sci_twiddles(int M) {
    auto w = [M](long long m) {
        const double a = -2.0 * M_PI * (double)m / (double)M;
        return make_float2((float)std::cos(a), (float)std::sin(a));
    };
    std::vector<float2> W(M);
    if (!sci_ct_size(M)) {
        for (int m = 0; m < M; ++m) W[m] = w(m);
        return W;
    }
    int off = 0;
    for (int ns = 1; ns < M; ns *= ct_radix(M / ns)) {
        const int R = ct_radix(M / ns);
        for (int r = 1; r < R; ++r)
            for (int k = 0; k < ns; ++k) W[off + (r - 1) * ns + k] = w(((long long)r * k * (M / (ns * R))) % M);
        off += ns * (R - 1);
    }
    return W;
}

cudaError_t sci_prepare(int M) {
    size_t sm = fft_smem_bytes(M);
    cudaError_t e = set_smem((const void*)sci_rows_kernel, sm);
    if (e != cudaSuccess) return e;
    e = set_smem((const void*)sci_cols_kernel, sm);
    if (e != cudaSuccess) return e;
#define MCAO_CT_PREP(n) \
    if (M >= n) {       \
        e = ct_prepare<n>(); \
        if (e != cudaSuccess) return e; \
    }
    MCAO_SCI_CT_SIZES(MCAO_CT_PREP)
#undef MCAO_CT_PREP
    return cudaSuccess;
}

size_t sci_smem_bytes(int M) { return fft_smem_bytes(M); }

cudaError_t launch_sci_rows(const SciLaunch& L, cudaStream_t s) {
#define MCAO_CT_ROWS(n) \
    if (L.M == n) return ct_rows<n>(L, s);
    MCAO_SCI_CT_SIZES(MCAO_CT_ROWS)
#undef MCAO_CT_ROWS
    size_t sm = fft_smem_bytes(L.M);
    sci_rows_kernel<<<dim3((unsigned)((L.N + kRowsPerBlock - 1) / kRowsPerBlock + 1), (unsigned)L.ctx.n_real), 256, sm, s>>>(L);
    return cudaGetLastError();
}

cudaError_t launch_sci_cols(const SciLaunch& L, cudaStream_t s) {
#define MCAO_CT_COLS(n) \
    if (L.M == n) return ct_cols<n>(L, s);
    MCAO_SCI_CT_SIZES(MCAO_CT_COLS)
#undef MCAO_CT_COLS
    size_t sm = fft_smem_bytes(L.M);
    sci_cols_kernel<<<dim3((unsigned)(L.M / kRowsPerBlock), (unsigned)L.ctx.n_real), 256, sm, s>>>(L);
    return cudaGetLastError();
}

namespace {

// (long-exposure, instantaneous) Strehl ratio of each science direction from its accumulators
__global__ void strehl_out_kernel(const SciAcc* acc, int n_sci, double* out) {
    const int q = blockIdx.x * blockDim.x + threadIdx.x;
    if (q >= n_sci) return;
    const SciAcc a = acc[q];
    out[2 * q] = a.n_sr ? a.sr_sum / (double)a.n_sr : 0.0;
    out[2 * q + 1] = a.sr_last;
}

// a step's readout into one slot of the device ring: the commands copied, the (long, last)
// Strehl ratios of each science direction formed as strehl_out_kernel does
__global__ void readout_kernel(const float* __restrict__ c, int n_cmd, const SciAcc* __restrict__ acc, int n_sci,
                               float* __restrict__ ring_c, double* __restrict__ ring_s) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n_cmd) ring_c[i] = c[i];
    if (i < n_sci) {
        const SciAcc a = acc[i];
        ring_s[2 * i] = a.n_sr ? a.sr_sum / (double)a.n_sr : 0.0;
        ring_s[2 * i + 1] = a.sr_last;
    }
}

}  // namespace

cudaError_t launch_readout(const float* c, int n_cmd, const SciAcc* acc, int n_sci, float* ring_c, double* ring_s,
                           cudaStream_t s) {
    const int n = std::max(n_cmd, n_sci);
    if (n > 0) readout_kernel<<<(n + 255) / 256, 256, 0, s>>>(c, n_cmd, acc, n_sci, ring_c, ring_s);
    return cudaGetLastError();
}

cudaError_t launch_strehl_out(const SciAcc* acc, int n_sci, double* out, cudaStream_t s) {
    if (n_sci > 0) strehl_out_kernel<<<(n_sci + 63) / 64, 64, 0, s>>>(acc, n_sci, out);
    return cudaGetLastError();
}

}  // namespace mcao
