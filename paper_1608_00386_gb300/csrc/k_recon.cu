// Reconstructor product and integrator ("The closed loop" of arXiv:1608.00386: slopes times the
// control matrix give differential coefficients added to the mirror commands; pure integrator):
//   Delta c = R s,   c <- c + g Delta c.
// R is float32 [n_cmd][n_slopes], far larger than L2, and is read exactly once per step, so the
// product is bound by HBM bandwidth.  The product is issued per slice of columns (one slice per
// wavefront sensor, so a slice can start as soon as its sensor's slopes exist) and split-K
// inside a slice: block (rb, kc) multiplies 32 rows by one column chunk of s held in shared
// memory; each warp streams four rows at a time with 16-byte evict-first loads and writes its
// row sums to a partial buffer [n_chunks][n_cmd].  A second kernel adds the partials in a fixed
// order (deterministic) and applies the gain.
#include "mcao_internal.h"

namespace mcao {

namespace {

constexpr int kKC = kReconChunk;
constexpr int kRowsPerWarp = 4;
constexpr int kWarps = 8;
constexpr int kRB = kRowsPerWarp * kWarps;
static_assert(kRB == kReconRowBlock, "row block");

__device__ __forceinline__ float dot4(float4 a, float4 b, float acc) {
    acc = fmaf(a.x, b.x, acc);
    acc = fmaf(a.y, b.y, acc);
    acc = fmaf(a.z, b.z, acc);
    return fmaf(a.w, b.w, acc);
}

__global__ void __launch_bounds__(256) recon_gemv_kernel(ReconLaunch L) {
    __shared__ float4 s_sh[kKC / 4];
    const int kc = blockIdx.y;
    const int c_begin = kc * L.kc;                 // column offset inside the slice
    int ncols = L.len - c_begin;
    if (ncols > L.kc) ncols = L.kc;
    const int n4 = (ncols + 3) / 4;                // R rows are zero-padded to a multiple of 4
    for (int i = threadIdx.x; i < n4; i += blockDim.x) {
        int c = c_begin + 4 * i;
        float4 v;
        v.x = (c + 0 < L.len) ? L.s[L.s0 + c + 0] : 0.0f;
        v.y = (c + 1 < L.len) ? L.s[L.s0 + c + 1] : 0.0f;
        v.z = (c + 2 < L.len) ? L.s[L.s0 + c + 2] : 0.0f;
        v.w = (c + 3 < L.len) ? L.s[L.s0 + c + 3] : 0.0f;
        s_sh[i] = v;
    }
    __syncthreads();

    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int row0 = blockIdx.x * kRB + warp * kRowsPerWarp;
    const size_t ld4 = (size_t)L.ld / 4;
    const float4* r0 = reinterpret_cast<const float4*>(L.R) + (size_t)row0 * ld4 + (L.col0 + c_begin) / 4;
    const float4* r1 = r0 + ld4;
    const float4* r2 = r1 + ld4;
    const float4* r3 = r2 + ld4;
    float a0 = 0.0f, a1 = 0.0f, a2 = 0.0f, a3 = 0.0f;
    int i = lane;
    // four float4 per row in flight per lane
    for (; i + 96 < n4; i += 128) {
        float4 x00 = __ldcs(r0 + i), x01 = __ldcs(r0 + i + 32), x02 = __ldcs(r0 + i + 64), x03 = __ldcs(r0 + i + 96);
        float4 x10 = __ldcs(r1 + i), x11 = __ldcs(r1 + i + 32), x12 = __ldcs(r1 + i + 64), x13 = __ldcs(r1 + i + 96);
        float4 x20 = __ldcs(r2 + i), x21 = __ldcs(r2 + i + 32), x22 = __ldcs(r2 + i + 64), x23 = __ldcs(r2 + i + 96);
        float4 x30 = __ldcs(r3 + i), x31 = __ldcs(r3 + i + 32), x32 = __ldcs(r3 + i + 64), x33 = __ldcs(r3 + i + 96);
        float4 s0 = s_sh[i], s1 = s_sh[i + 32], s2 = s_sh[i + 64], s3 = s_sh[i + 96];
        a0 = dot4(x00, s0, a0); a0 = dot4(x01, s1, a0); a0 = dot4(x02, s2, a0); a0 = dot4(x03, s3, a0);
        a1 = dot4(x10, s0, a1); a1 = dot4(x11, s1, a1); a1 = dot4(x12, s2, a1); a1 = dot4(x13, s3, a1);
        a2 = dot4(x20, s0, a2); a2 = dot4(x21, s1, a2); a2 = dot4(x22, s2, a2); a2 = dot4(x23, s3, a2);
        a3 = dot4(x30, s0, a3); a3 = dot4(x31, s1, a3); a3 = dot4(x32, s2, a3); a3 = dot4(x33, s3, a3);
    }
    for (; i < n4; i += 32) {
        float4 s0 = s_sh[i];
        a0 = dot4(__ldcs(r0 + i), s0, a0);
        a1 = dot4(__ldcs(r1 + i), s0, a1);
        a2 = dot4(__ldcs(r2 + i), s0, a2);
        a3 = dot4(__ldcs(r3 + i), s0, a3);
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        a0 += __shfl_xor_sync(0xffffffffu, a0, o);
        a1 += __shfl_xor_sync(0xffffffffu, a1, o);
        a2 += __shfl_xor_sync(0xffffffffu, a2, o);
        a3 += __shfl_xor_sync(0xffffffffu, a3, o);
    }
    if (lane == 0) {
        float* p = L.partial + (size_t)(L.chunk0 + kc) * L.n_cmd;
        if (row0 + 0 < L.n_cmd) p[row0 + 0] = a0;
        if (row0 + 1 < L.n_cmd) p[row0 + 1] = a1;
        if (row0 + 2 < L.n_cmd) p[row0 + 2] = a2;
        if (row0 + 3 < L.n_cmd) p[row0 + 3] = a3;
    }
}

__global__ void recon_reduce_kernel(ReduceLaunch L) {
    int row = blockIdx.x * blockDim.x + threadIdx.x;
    if (row == 0 && L.st) L.st->k_next = L.st->k + 1;
    if (row >= L.n_cmd) return;
    float acc = 0.0f;
    for (int kc = 0; kc < L.n_chunks; ++kc) acc += L.partial[(size_t)kc * L.n_cmd + row];
    L.c[row] = fmaf(L.gain, acc, L.c[row]);
}

}  // namespace

cudaError_t launch_recon(const ReconLaunch& L, cudaStream_t s) {
    if (L.n_cmd <= 0 || L.len <= 0) return cudaSuccess;
    dim3 grid((unsigned)(L.rows_pad / kRB), (unsigned)((L.len + L.kc - 1) / L.kc));
    recon_gemv_kernel<<<grid, 256, 0, s>>>(L);
    return cudaGetLastError();
}

cudaError_t launch_recon_reduce(const ReduceLaunch& L, cudaStream_t s) {
    int n = L.n_cmd > 0 ? L.n_cmd : 1;
    recon_reduce_kernel<<<(unsigned)((n + 255) / 256), 256, 0, s>>>(L);
    return cudaGetLastError();
}

}  // namespace mcao
