// Allocation-free variant of the reconstructor update c <- c + gain R s
// (mcao_reconstruct_noalloc in include/mcao.h).
//
// The split-K product needs scratch space for one partial sum per (column chunk, row).  The
// closed-loop simulation allocates it with cudaMalloc when the reconstructor is loaded; this
// entry point instead keeps it in a fixed file-scope device array, so a caller that must not
// allocate device memory can still run the update on buffers it already owns.  The array is
// created when the library is loaded on a device and lives until the process exits.
#include <cuda_runtime.h>

#include <cmath>
#include <cstdarg>
#include <cstdint>
#include <cstdio>
#include <mutex>

#include "../../include/mcao.h"

namespace {

constexpr long long kScratchFloats = 1ll << 19;   // 524288 partial sums = 2 MiB
constexpr int kChunk = 4096;                       // slope columns per block (at most)
constexpr int kRowsPerWarp = 4;
constexpr int kRowBlock = 32;
constexpr int kMaxDevices = 64;

static __device__ __align__(256) float g_noalloc_partial[kScratchFloats];

__device__ __forceinline__ float dot4(float4 a, float4 b, float acc) {
    acc = fmaf(a.x, b.x, acc);
    acc = fmaf(a.y, b.y, acc);
    acc = fmaf(a.z, b.z, acc);
    return fmaf(a.w, b.w, acc);
}

// Block (rb, kc): rows [32 rb, 32 rb + 32) times columns [kc kc_len, ...) of R, row sums to
// partial[kc][row].  Rows past n_cmd re-read the last row (their sums are not stored), so the
// caller's R needs no row padding.  Only columns below n_slopes are read: the last chunk's
// ragged tail (n_slopes not a multiple of 4) is loaded element by element, so whatever the
// caller keeps in the padding columns n_slopes..ld-1 (even NaN) never enters a sum.
__global__ void __launch_bounds__(256) noalloc_gemv(const float* __restrict__ R, int n_cmd, int n_slopes, int ld,
                                                    const float* __restrict__ s, float* __restrict__ partial,
                                                    int kc_len) {
    __shared__ float4 s_sh[kChunk / 4];
    const int kc = blockIdx.y;
    const int c_begin = kc * kc_len;
    int ncols = n_slopes - c_begin;
    if (ncols > kc_len) ncols = kc_len;
    const int n4 = (ncols + 3) / 4;
    const int nfull = ncols / 4;                       // whole 16-byte vectors inside the chunk
    for (int i = threadIdx.x; i < n4; i += blockDim.x) {
        int c = c_begin + 4 * i;
        float4 v;
        v.x = (c + 0 < n_slopes) ? s[c + 0] : 0.0f;
        v.y = (c + 1 < n_slopes) ? s[c + 1] : 0.0f;
        v.z = (c + 2 < n_slopes) ? s[c + 2] : 0.0f;
        v.w = (c + 3 < n_slopes) ? s[c + 3] : 0.0f;
        s_sh[i] = v;
    }
    __syncthreads();
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int row0 = blockIdx.x * kRowBlock + warp * kRowsPerWarp;
    const size_t ld4 = (size_t)ld / 4;
    const float4* rp[kRowsPerWarp];
#pragma unroll
    for (int q = 0; q < kRowsPerWarp; ++q) {
        int row = min(row0 + q, n_cmd - 1);
        rp[q] = reinterpret_cast<const float4*>(R) + (size_t)row * ld4 + c_begin / 4;
    }
    float acc[kRowsPerWarp] = {0.0f, 0.0f, 0.0f, 0.0f};
    for (int i = lane; i < nfull; i += 32) {
        float4 sv = s_sh[i];
#pragma unroll
        for (int q = 0; q < kRowsPerWarp; ++q) acc[q] = dot4(__ldcs(rp[q] + i), sv, acc[q]);
    }
    if (nfull < n4 && lane == (nfull & 31)) {          // 1-3 columns left, read one by one
        const float4 sv = s_sh[nfull];
        const int rem = ncols - 4 * nfull;
#pragma unroll
        for (int q = 0; q < kRowsPerWarp; ++q) {
            const float* rq = reinterpret_cast<const float*>(rp[q] + nfull);
            acc[q] = fmaf(rq[0], sv.x, acc[q]);
            if (rem > 1) acc[q] = fmaf(rq[1], sv.y, acc[q]);
            if (rem > 2) acc[q] = fmaf(rq[2], sv.z, acc[q]);
        }
    }
#pragma unroll
    for (int q = 0; q < kRowsPerWarp; ++q) {
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) acc[q] += __shfl_xor_sync(0xffffffffu, acc[q], o);
    }
    if (lane == 0) {
        float* p = partial + (size_t)kc * n_cmd;
#pragma unroll
        for (int q = 0; q < kRowsPerWarp; ++q)
            if (row0 + q < n_cmd) p[row0 + q] = acc[q];
    }
}

__global__ void noalloc_reduce(const float* __restrict__ partial, int n_chunks, int n_cmd, float* __restrict__ c,
                               float gain) {
    int row = blockIdx.x * blockDim.x + threadIdx.x;
    if (row >= n_cmd) return;
    float acc = 0.0f;
    for (int kc = 0; kc < n_chunks; ++kc) acc += partial[(size_t)kc * n_cmd + row];
    c[row] = fmaf(gain, acc, c[row]);
}

std::mutex g_mu;
float* g_scratch[kMaxDevices] = {nullptr};

mcao_status report(char* err, size_t err_len, mcao_status st, const char* fmt, ...) {
    if (err && err_len) {
        va_list ap;
        va_start(ap, fmt);
        vsnprintf(err, err_len, fmt, ap);
        va_end(ap);
    }
    return st;
}

}  // namespace

extern "C" mcao_status mcao_reconstruct_noalloc(const float* R, int n_cmd, int n_slopes, int ld, const float* s,
                                                float* c, float gain, void* stream, char* err, size_t err_len) {
    if (err && err_len) err[0] = '\0';
    if (!R || !s || !c) return report(err, err_len, MCAO_E_INVALID_ARG, "R, s and c must be device pointers");
    if (n_cmd < 1 || n_slopes < 1 || ld < n_slopes || ld % 4 != 0)
        return report(err, err_len, MCAO_E_INVALID_ARG, "need n_cmd >= 1, n_slopes >= 1, ld >= n_slopes, ld %% 4 == 0");
    if (((uintptr_t)R) % 16 != 0) return report(err, err_len, MCAO_E_INVALID_ARG, "R must be 16-byte aligned");
    if (!std::isfinite(gain)) return report(err, err_len, MCAO_E_INVALID_ARG, "gain must be finite");
    int n_chunks = (n_slopes + kChunk - 1) / kChunk;
    int kc_len = (n_slopes + n_chunks - 1) / n_chunks;
    kc_len = (kc_len + 3) / 4 * 4;
    n_chunks = (n_slopes + kc_len - 1) / kc_len;
    if ((long long)n_chunks * n_cmd > kScratchFloats)
        return report(err, err_len, MCAO_E_SHAPE,
                      "n_cmd x column chunks = %d x %d exceeds the %lld-float scratch of the allocation-free update",
                      n_cmd, n_chunks, kScratchFloats);
    if (n_chunks > 65535)
        return report(err, err_len, MCAO_E_SHAPE, "%d column chunks exceed the launch's 65535 grid rows", n_chunks);
    // An error left pending by earlier work of the caller would otherwise be reported as this
    // call's launch failure: name it as such and launch nothing.
    cudaError_t e = cudaPeekAtLastError();
    if (e != cudaSuccess)
        return report(err, err_len, MCAO_E_CUDA, "a CUDA error was pending before this call: %s",
                      cudaGetErrorString(e));
    int dev = 0;
    e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return report(err, err_len, MCAO_E_CUDA, "cudaGetDevice: %s", cudaGetErrorString(e));
    if (dev < 0 || dev >= kMaxDevices) return report(err, err_len, MCAO_E_UNSUPPORTED, "device %d out of range", dev);
    float* scratch = nullptr;
    {
        std::lock_guard<std::mutex> lock(g_mu);
        if (!g_scratch[dev]) {
            void* p = nullptr;
            e = cudaGetSymbolAddress(&p, g_noalloc_partial);
            if (e != cudaSuccess)
                return report(err, err_len, MCAO_E_CUDA, "cudaGetSymbolAddress: %s", cudaGetErrorString(e));
            g_scratch[dev] = static_cast<float*>(p);
        }
        scratch = g_scratch[dev];
    }
    cudaStream_t st = (cudaStream_t)stream;
    dim3 grid((unsigned)((n_cmd + kRowBlock - 1) / kRowBlock), (unsigned)n_chunks);
    noalloc_gemv<<<grid, 256, 0, st>>>(R, n_cmd, n_slopes, ld, s, scratch, kc_len);
    e = cudaGetLastError();
    if (e != cudaSuccess) return report(err, err_len, MCAO_E_CUDA, "product launch: %s", cudaGetErrorString(e));
    noalloc_reduce<<<(unsigned)((n_cmd + 255) / 256), 256, 0, st>>>(scratch, n_chunks, n_cmd, c, gain);
    e = cudaGetLastError();
    if (e != cudaSuccess) return report(err, err_len, MCAO_E_CUDA, "reduction launch: %s", cudaGetErrorString(e));
    return MCAO_OK;
}
