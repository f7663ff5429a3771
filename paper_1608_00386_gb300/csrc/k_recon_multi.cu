// Reconstructor product for up to 16 realizations sharing R ("The closed loop": slopes times the
// control matrix, here for a batch of independent realizations): D[r][i] = sum_j R[i][j] s_r[j].
//
// R is held column-major, [ld][rows_pad] (float32 or bfloat16), and streamed once per step: a
// warp item is 128 rows (4 per lane) x 1024 columns; per column each lane copies its 4 rows
// (16 bytes float32, 8 bytes bfloat16) asynchronously into its own shared-memory slot, three
// groups of 8 columns ahead of the multiply-adds (cp.async with per-thread completion groups),
// the group's slopes of every realization (from a transposed copy S_t[j][r], 16 floats per
// column, zero past n_real) travel in the same groups, one 16-byte copy per lane, and are read
// back as shared-memory broadcasts; each lane accumulates 4 rows x 16 realizations in float32
// with packed FMAs.  Reading the slopes through L1 instead left every column waiting on L2: the
// ring leaves little L1, and each warp walks its own 64 KB of slopes.  Items write
// split-K partials [chunk][16][n_cmd]; a second kernel sums them in a fixed order, so the
// result does not depend on which warp took which item.
#include <type_traits>

#include "mcao_internal.h"

namespace mcao {

namespace {

constexpr int kMRows = 128;    // rows per item (4 per lane)
constexpr int kMCols = 1024;   // columns per item
constexpr int kMUnroll = 8;    // columns whose loads are in flight together
constexpr int kMB = kMultiRhs; // realizations per pass

// packed float32 pairs held in 64-bit registers: packing once per operand and accumulating in
// place keeps the packed multiply-adds free of per-call register moves
__device__ __forceinline__ unsigned long long pack2(float x, float y) {
    unsigned long long d;
    asm("mov.b64 %0, {%1, %2};" : "=l"(d) : "f"(x), "f"(y));
    return d;
}
__device__ __forceinline__ void ffma2_acc(unsigned long long& acc, unsigned long long a, unsigned long long b) {
    asm("fma.rn.f32x2 %0, %1, %2, %0;" : "+l"(acc) : "l"(a), "l"(b));
}
__device__ __forceinline__ float2 unpack2(unsigned long long v) {
    float2 r;
    asm("mov.b64 {%0, %1}, %2;" : "=f"(r.x), "=f"(r.y) : "l"(v));
    return r;
}

// asynchronous copy of one lane's rows of a column into its private shared-memory slot
// (16 bytes float32, 8 bytes bfloat16; src_bytes = 0 fills zeros without reading)
template <bool BF16>
__device__ __forceinline__ void copy_rows(void* dst, const void* src, bool valid) {
    const uint32_t d = (uint32_t)__cvta_generic_to_shared(dst);
    if constexpr (BF16)
        asm volatile("cp.async.ca.shared.global [%0], [%1], 8, %2;" ::"r"(d), "l"(src), "r"(valid ? 8 : 0) : "memory");
    else
        asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;" ::"r"(d), "l"(src), "r"(valid ? 16 : 0) : "memory");
}
__device__ __forceinline__ void copy_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
template <int N>
__device__ __forceinline__ void copy_wait() { asm volatile("cp.async.wait_group %0;" ::"n"(N) : "memory"); }

constexpr int kMStages = 3;   // column groups in flight per warp
constexpr int kMWarps = 8;

template <bool BF16>
struct MultiRing {
    // per warp, stage, column of the group and lane: that lane's 4 rows of the column
    typename std::conditional<BF16, uint2, float4>::type v[kMWarps][kMStages][kMUnroll][32];
    // per warp and stage: the group's slopes S_t[j][0..16) (one 16-byte copy per lane)
    float4 s[kMWarps][kMStages][kMUnroll * kMB / 4];
};
static_assert(kMUnroll * kMB / 4 == 32, "one slope vector per lane and group");

template <bool BF16>
__global__ void __launch_bounds__(kMWarps * 32) recon_multi_kernel(MultiLaunch L) {
    extern __shared__ __align__(16) unsigned char multi_raw[];
    MultiRing<BF16>& ring = *reinterpret_cast<MultiRing<BF16>*>(multi_raw);
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int n_warps = (gridDim.x * blockDim.x) >> 5;
    const int n_rb = (L.n_cmd + kMRows - 1) / kMRows;
    const int n_kc = (L.K + kMCols - 1) / kMCols;
    const float4* S4 = reinterpret_cast<const float4*>(L.s_t);
    const int esz = BF16 ? 2 : 4;
    const unsigned char* Rb = reinterpret_cast<const unsigned char*>(L.R);
    for (int item = (int)((blockIdx.x * blockDim.x + threadIdx.x) >> 5); item < n_rb * n_kc; item += n_warps) {
        const int kc = item / n_rb, rb = item - kc * n_rb;
        const int row0 = rb * kMRows + 4 * lane;
        const bool live = row0 < L.rows_pad;   // rows_pad is a multiple of 4
        const int c0 = kc * kMCols, c1 = min(L.K, c0 + kMCols);
        const int n_groups = (c1 - c0 + kMUnroll - 1) / kMUnroll;
        auto issue = [&](int g) {
            if (g < n_groups) {
                const int st = g % kMStages;
#pragma unroll
                for (int u = 0; u < kMUnroll; ++u) {
                    const int j = c0 + g * kMUnroll + u;
                    const bool ok = live && j < c1;
                    const long long off = ok ? ((long long)j * L.rows_pad + row0) * esz : 0;
                    copy_rows<BF16>(&ring.v[warp][st][u][lane], Rb + off, ok);
                }
                const int js = c0 + g * kMUnroll + lane / (kMB / 4);   // column of this lane's slope vector
                const bool oks = js < c1;
                const uint32_t d = (uint32_t)__cvta_generic_to_shared(&ring.s[warp][st][lane]);
                asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;" ::"r"(d),
                             "l"(S4 + (oks ? (long long)c0 * (kMB / 4) + (long long)g * (kMUnroll * kMB / 4) + lane : 0)),
                             "r"(oks ? 16 : 0)
                             : "memory");
            }
            copy_commit();   // an empty group past the end keeps the wait count uniform
        };
        unsigned long long acc[4][kMB / 2];
#pragma unroll
        for (int q = 0; q < 4; ++q)
#pragma unroll
            for (int b = 0; b < kMB / 2; ++b) acc[q][b] = 0ull;   // (+0.0f, +0.0f)
#pragma unroll
        for (int g = 0; g < kMStages - 1; ++g) issue(g);
        for (int g = 0; g < n_groups; ++g) {
            __syncwarp();   // every lane has read the slot that the next copy refills
            issue(g + kMStages - 1);
            copy_wait<kMStages - 1>();   // this lane's copies of group g have landed
            __syncwarp();                // and every lane's (the slope vectors are shared)
            const int st = g % kMStages;
#pragma unroll
            for (int u = 0; u < kMUnroll; ++u) {
                const int j = c0 + g * kMUnroll + u;
                if (j >= c1) break;
                float4 r;
                if constexpr (BF16) {
                    const uint2 w = ring.v[warp][st][u][lane];
                    r = make_float4(__uint_as_float(w.x << 16), __uint_as_float(w.x & 0xffff0000u),
                                    __uint_as_float(w.y << 16), __uint_as_float(w.y & 0xffff0000u));
                } else {
                    r = ring.v[warp][st][u][lane];
                }
                const unsigned long long rp[4] = {pack2(r.x, r.x), pack2(r.y, r.y), pack2(r.z, r.z), pack2(r.w, r.w)};
#pragma unroll
                for (int b4 = 0; b4 < kMB / 4; ++b4) {
                    const float4 sv = ring.s[warp][st][u * (kMB / 4) + b4];
                    const unsigned long long s01 = pack2(sv.x, sv.y), s23 = pack2(sv.z, sv.w);
#pragma unroll
                    for (int q = 0; q < 4; ++q) {
                        ffma2_acc(acc[q][2 * b4], rp[q], s01);
                        ffma2_acc(acc[q][2 * b4 + 1], rp[q], s23);
                    }
                }
            }
        }
        copy_wait<0>();   // nothing of this item is left in flight before the slots are reused
        __syncwarp();
        if (!live) continue;
        float* out = L.partial + (long long)kc * kMB * L.n_cmd;
#pragma unroll
        for (int q = 0; q < 4; ++q) {
            const int row = row0 + q;
            if (row >= L.n_cmd) continue;
#pragma unroll
            for (int b = 0; b < kMB / 2; ++b) {
                const float2 v = unpack2(acc[q][b]);
                out[(long long)(2 * b) * L.n_cmd + row] = v.x;
                out[(long long)(2 * b + 1) * L.n_cmd + row] = v.y;
            }
        }
    }
}

// S_t[j][r] = slopes of realization r at padded column j (zero for r >= n_real)
__global__ void slopes_t_kernel(const float* slopes_pad, int n_real, int K, int pad_stride, float* s_t) {
    const long long total = (long long)K * kMB;
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < total; i += (long long)gridDim.x * blockDim.x) {
        const int j = (int)(i / kMB), r = (int)(i - (long long)j * kMB);
        s_t[i] = r < n_real ? slopes_pad[(long long)r * pad_stride + j] : 0.0f;
    }
}

// out[r][i] = alpha sum_kc partial[kc][r][i] + beta out[r][i] (beta = 0: out not read)
__global__ void multi_reduce_kernel(const float* partial, int n_kc, int n_real, int n_cmd, float alpha, float beta,
                                    float* out) {
    const long long total = (long long)n_real * n_cmd;
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < total; i += (long long)gridDim.x * blockDim.x) {
        const int r = (int)(i / n_cmd), row = (int)(i - (long long)r * n_cmd);
        float s = 0.0f;
        for (int kc = 0; kc < n_kc; ++kc) s += partial[((long long)kc * kMB + r) * n_cmd + row];
        out[i] = beta == 0.0f ? alpha * s : fmaf(alpha, s, beta * out[i]);
    }
}

}  // namespace

int multi_chunks(int K) { return (K + kMCols - 1) / kMCols; }

cudaError_t multi_prepare() {
    cudaError_t e = cudaFuncSetAttribute(recon_multi_kernel<false>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)sizeof(MultiRing<false>));
    if (e == cudaSuccess)
        e = cudaFuncSetAttribute(recon_multi_kernel<true>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 (int)sizeof(MultiRing<true>));
    return e;
}

cudaError_t launch_recon_multi(const MultiLaunch& L, int n_real, int pad_stride, const float* slopes_pad, float alpha,
                               float beta, float* out, int sm_count, int blocks_per_sm, cudaStream_t s) {
    if (n_real < 1 || n_real > kMB) return cudaErrorInvalidValue;
    slopes_t_kernel<<<256, 256, 0, s>>>(slopes_pad, n_real, L.K, pad_stride, L.s_t);
    const int items = ((L.n_cmd + kMRows - 1) / kMRows) * multi_chunks(L.K);
    int blocks = (items + kMWarps - 1) / kMWarps;
    const int cap = (blocks_per_sm > 0 ? blocks_per_sm : 2) * sm_count;   // at most two resident per SM
    if (blocks > cap) blocks = cap;
    if (L.bf16)
        recon_multi_kernel<true><<<blocks, kMWarps * 32, sizeof(MultiRing<true>), s>>>(L);
    else
        recon_multi_kernel<false><<<blocks, kMWarps * 32, sizeof(MultiRing<false>), s>>>(L);
    multi_reduce_kernel<<<(n_real * L.n_cmd + 255) / 256, 256, 0, s>>>(L.partial, multi_chunks(L.K), n_real, L.n_cmd,
                                                                       alpha, beta, out);
    return cudaGetLastError();
}

}  // namespace mcao
