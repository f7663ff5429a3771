// DM surfaces (Gaussian influence functions, "Influence function and modal base" of
// arXiv:1608.00386): S = sum_j c_j exp(-|x - x_j|^2 / 2 sigma^2), with exp(-pitch^2/2 sigma^2)
// equal to the coupling.  The Gaussian factorises, so S = Gy C Gx^T exactly.  One block per
// 32 x 32 tile of the surface: the tile's actuator sub-grid C (rows and columns whose weight on
// the tile is at least 1e-10; dropped terms are below float rounding of the surface), the
// matching Gx and Gy rows and T = C Gx^T are staged in shared memory, then S = Gy T.  A
// translated or magnified DM has its transform folded into Gx and Gy; a rotated one evaluates
// every sample against the actuators around its position in the DM's own frame.
#include "mcao_internal.h"

namespace mcao {

namespace {

constexpr int kT = kDmTile;
constexpr int kB = kDmMaxBand;

__global__ void __launch_bounds__(256) dm_surface_kernel(DmLaunch L) {
    __shared__ float s_C[kB][kB + 1];
    __shared__ float s_Gx[kT][kB + 1];
    __shared__ float s_Gy[kT][kB + 1];
    __shared__ float s_T[kB][kT];
    if (blockIdx.x == 0 && blockIdx.y == 0) {
        if (threadIdx.x == 0 && L.st) L.st->k = L.st->k_next;
        for (int i = threadIdx.x; i < L.n_work; i += blockDim.x) L.work[i] = 0u;
        for (int i = threadIdx.x; i < L.n_rq; i += blockDim.x) L.rq_done[i] = 0u;
    }
    const int real = blockIdx.y;   // realization
    const float* cmd = L.c + (long long)real * L.n_cmd;
    int t = blockIdx.x;
    int m = 0;
    while (m + 1 < L.n_dm && t >= L.tile_start[m + 1]) ++m;
    const DmDesc& d = L.desc[m];
    t -= L.tile_start[m];
    const int n = d.surf_n;
    const int ty_i = t / d.tiles_x, tx_i = t % d.tiles_x;
    const int j0 = ty_i * kT, i0 = tx_i * kT;
    if (d.general) {
        // rotated DM: each sample q = R(-rot)((x, y) - shift) / mag weighs the actuators within rc
        // pitches directly
        const float c0 = 0.5f * (float)(n - 1), ca = 0.5f * (float)(d.nx - 1), cb = 0.5f * (float)(d.ny - 1);
        for (int q = threadIdx.x; q < kT * kT; q += blockDim.x) {
            const int i = i0 + (q & (kT - 1)), j = j0 + q / kT;
            if (i >= n || j >= n) continue;
            const float x = ((float)i - c0) * d.dx - d.shx, y = ((float)j - c0) * d.dx - d.shy;
            const float ua = (d.cr * x + d.sr * y) * d.inv_mag / d.pitch + ca;
            const float ub = (-d.sr * x + d.cr * y) * d.inv_mag / d.pitch + cb;
            const int a0 = max(0, (int)ceilf(ua - d.rc)), a1 = min(d.nx - 1, (int)floorf(ua + d.rc));
            const int b0 = max(0, (int)ceilf(ub - d.rc)), b1 = min(d.ny - 1, (int)floorf(ub + d.rc));
            float acc = 0.0f;
            for (int b = b0; b <= b1; ++b) {
                const float dy = (ub - (float)b) * d.pitch;
                float row = 0.0f;
                for (int a = a0; a <= a1; ++a) {
                    const int idx = L.act_map[d.map_off + (long long)b * d.nx + a];
                    if (idx < 0) continue;
                    const float dxa = (ua - (float)a) * d.pitch;
                    row = fmaf(cmd[idx], expf(-dxa * dxa * d.inv2s2), row);
                }
                acc = fmaf(expf(-dy * dy * d.inv2s2), row, acc);
            }
            L.surf[real * L.surf_stride + d.surf_off + (long long)j * n + i] = acc;
        }
        return;
    }
    const int2 bx = L.band[d.tband_x + tx_i], by = L.band[d.tband_y + ty_i];
    const int na = bx.y - bx.x, nb = by.y - by.x;
    const int tid = threadIdx.x;
    // commands of the actuator sub-grid, and the Gaussian weights of the tile's rows / columns
    // (2-D thread mappings: no division by the runtime band sizes)
    const int lane = tid & 31, wid = tid >> 5;
    for (int bb = wid; bb < nb; bb += 8)
        for (int aa = lane; aa < na; aa += 32) {
            int idx = L.act_map[d.map_off + (long long)(by.x + bb) * d.nx + bx.x + aa];
            s_C[bb][aa] = (idx >= 0) ? cmd[idx] : 0.0f;
        }
    for (int ii = tid >> 3; ii < kT; ii += 32) {
        const int i = i0 + ii;
        for (int aa = tid & 7; aa < na; aa += 8)
            s_Gx[ii][aa] = (i < n) ? L.g[d.gx_off + (long long)i * d.nx + bx.x + aa] : 0.0f;
        const int j = j0 + ii;
        for (int bb = tid & 7; bb < nb; bb += 8)
            s_Gy[ii][bb] = (j < n) ? L.g[d.gy_off + (long long)j * d.ny + by.x + bb] : 0.0f;
    }
    __syncthreads();
    // T[bb][ii] = sum_aa C[bb][aa] Gx[ii][aa]
    for (int bb = wid; bb < nb; bb += 8) {
        float acc = 0.0f;
        for (int aa = 0; aa < na; ++aa) acc = fmaf(s_C[bb][aa], s_Gx[lane][aa], acc);
        s_T[bb][lane] = acc;
    }
    __syncthreads();
    // S[jj][ii] = sum_bb Gy[jj][bb] T[bb][ii]; thread -> column ii, rows 4 ty .. 4 ty + 3
    const int ii = tid & 31, ty = tid >> 5;
    float acc0 = 0.0f, acc1 = 0.0f, acc2 = 0.0f, acc3 = 0.0f;
    for (int bb = 0; bb < nb; ++bb) {
        const float tv = s_T[bb][ii];
        acc0 = fmaf(s_Gy[ty * 4 + 0][bb], tv, acc0);
        acc1 = fmaf(s_Gy[ty * 4 + 1][bb], tv, acc1);
        acc2 = fmaf(s_Gy[ty * 4 + 2][bb], tv, acc2);
        acc3 = fmaf(s_Gy[ty * 4 + 3][bb], tv, acc3);
    }
    const int i = i0 + ii;
    if (i < n) {
        float* out = L.surf + real * L.surf_stride + d.surf_off + i;
        const float acc[4] = {acc0, acc1, acc2, acc3};
#pragma unroll
        for (int r = 0; r < 4; ++r) {
            const int j = j0 + ty * 4 + r;
            if (j < n) out[(long long)j * n] = acc[r];
        }
    }
}

__global__ void begin_step_kernel(StepState* st, unsigned int* work, int n_work, unsigned int* rq_done, int n_rq) {
    if (threadIdx.x == 0 && st) st->k = st->k_next;
    for (int i = threadIdx.x; i < n_work; i += blockDim.x) work[i] = 0u;
    for (int i = threadIdx.x; i < n_rq; i += blockDim.x) rq_done[i] = 0u;
}

}  // namespace

cudaError_t launch_dm_surfaces(const DmLaunch& L, cudaStream_t s) {
    if (L.n_dm <= 0) return launch_begin_step(L.st, L.work, L.n_work, L.rq_done, L.n_rq, s);
    dm_surface_kernel<<<dim3((unsigned)L.tile_start[L.n_dm], (unsigned)(L.n_real > 0 ? L.n_real : 1)), 256, 0, s>>>(L);
    return cudaGetLastError();
}

cudaError_t launch_begin_step(StepState* st, unsigned int* work, int n_work, unsigned int* rq_done, int n_rq,
                              cudaStream_t s) {
    if (!st && n_work <= 0 && n_rq <= 0) return cudaSuccess;
    begin_step_kernel<<<1, 128, 0, s>>>(st, work, n_work, rq_done, n_rq);
    return cudaGetLastError();
}

}  // namespace mcao
