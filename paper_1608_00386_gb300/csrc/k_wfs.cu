// Shack-Hartmann wavefront sensing of the residual phase ("The closed loop" of
// arXiv:1608.00386: the WFS modules compute X and Y slopes from the open-loop wavefront minus
// the DMs), fused per subaperture: cone-beam propagation of every layer and DM, field
// A exp(i phi), spot formation, sodium elongation, binning, flux normalisation, photon and read
// noise, centre of gravity minus the reference slopes.
//
// Spot formation.  The defining computation is: zero-pad the n x n field to N x N, I = |FFT2|^2,
// elongate by FFT2(I) * OTF -> IFFT2, fftshift, bin b x b.  Two kernels compute exactly that
// result by cheaper routes:
//  * autocorrelation route (8 x 8 subapertures, with or without elongation): FFT2(I)(u) equals
//    N^2 ACF(u), ACF(u) = sum_y E(y - u) conj(E(y)), nonzero only for |u| <= n-1 < N/2.  Shift
//    by N/2 and b x b binning are, in the frequency domain, the factor
//    h(u) = (-1)^u sum_{t<b} e^{2 pi i u t/N} per axis followed by an (N/b)-point inverse DFT
//    of the lags: B[m] = sum_u ACF(u) OTF(u) h(ux) h(uy) e^{2 pi i u.m / n_det} (up to a
//    constant that the flux normalisation removes).  With rows r and columns a, b,
//    ACF(ux, uy) = sum_a M_uy[a][a + ux], M_uy[a][b] = sum_r E[r][a] conj(E[r + uy][b]): each
//    lane keeps three columns of E in registers and forms two entries of every M_uy.  One warp
//    per subaperture; no N x N array is formed.
//  * FFT route (large subapertures without elongation, e.g. 2 x 2 low-order sensors):
//    radix-4 Stockham FFTs of the padded field in shared memory, |.|^2, shift and bin; one
//    1024-thread block per subaperture.
#include <math.h>

#include "device_common.cuh"
#include "mcao_internal.h"

namespace mcao {

namespace {

constexpr float kPi = 3.14159265358979323846f;

// ------------------------------------------------------------------------------------------
// autocorrelation route: one warp per 8 x 8 subaperture, 8 warps per block
// ------------------------------------------------------------------------------------------
template <int NFFT, int NBIN>
__global__ void __launch_bounds__(256) wfs_acf_kernel(WfsLaunch L) {
    constexpr int NPX = 8;
    constexpr int ND = NFFT / NBIN;
    constexpr int NL = 2 * NPX - 1;
    constexpr int PIX_PER_LANE = (ND * ND + 31) / 32;
    constexpr int Y_PER_LANE = (NPX * ND + 31) / 32;
    __shared__ AxisEnt s_ex[8][kMaxEntries * NPX];
    __shared__ AxisEnt s_ey[8][kMaxEntries * NPX];
    __shared__ float2 s_E[8][NPX * NPX];
    __shared__ float2 s_M[8][NPX * NPX];
    __shared__ float2 s_P[8][NPX * NL];
    __shared__ float2 s_Y[8][NPX * ND];
    __shared__ float2 s_tw[8][ND];
    __shared__ float s_recip[8][65];

    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int sub = blockIdx.x * 8 + warp;
    if (sub >= L.n_subaps) return;  // warp-uniform; the kernel uses warp-level sync only
    const SubapDev sd = L.subaps[sub];
    const WfsDev& w = L.ctx.wfs[sd.wfs];
    const int i0 = sd.sx * NPX, j0 = sd.sy * NPX;
    const int n_grids = L.ctx.n_grids;
    const GridView* V = L.ctx.views + (long long)sd.wfs * n_grids;
    const long long k = L.ctx.st->k;

    tile_entries(V, n_grids, k, i0, j0, NPX, s_ex[warp], s_ey[warp], lane, 32);
    if (lane < ND) s_tw[warp][lane] = w.tw[lane];
    if (L.ctx.noise) fill_recip(s_recip[warp], lane, 32);
    __syncwarp();

    // field E = A exp(i (scale phi - pi (x + y) / N)): lane -> column x, rows y and y + 4
    const float scale = w.scale;
    {
        const int x = lane & 7;
#pragma unroll
        for (int hh = 0; hh < 2; ++hh) {
            const int y = (lane >> 3) + 4 * hh;
            float phi = tile_phase(V, n_grids, s_ex[warp], s_ey[warp], NPX, x, y);
            float a = __ldg(w.amp + (long long)(j0 + y) * w.N + i0 + x);
            float arg = scale * phi - kPi * (float)(x + y) / (float)NFFT;
            float sn, cs;
            sincosf(arg, &sn, &cs);
            s_E[warp][y * NPX + x] = make_float2(a * cs, a * sn);
        }
    }
    __syncwarp();

    // columns a, b0, b1 of E in registers
    const int ca_i = lane >> 2, cb_i = lane & 3;
    float2 ca[NPX], cb0[NPX], cb1[NPX];
#pragma unroll
    for (int r = 0; r < NPX; ++r) {
        ca[r] = s_E[warp][r * NPX + ca_i];
        cb0[r] = s_E[warp][r * NPX + cb_i];
        cb1[r] = s_E[warp][r * NPX + cb_i + 4];
    }
    float2 hx = make_float2(0.0f, 0.0f);
    if (lane < NL) hx = w.h[lane];  // h(ux), ux = lane - 7
    const int ux = lane - (NPX - 1);

#pragma unroll
    for (int uy = 0; uy < NPX; ++uy) {
        float m0r = 0.0f, m0i = 0.0f, m1r = 0.0f, m1i = 0.0f;
#pragma unroll
        for (int r = 0; r + uy < NPX; ++r) {
            // ca[r] conj(cb[r + uy])
            float2 a = ca[r], b0 = cb0[r + uy], b1 = cb1[r + uy];
            m0r = fmaf(a.x, b0.x, fmaf(a.y, b0.y, m0r));
            m0i = fmaf(a.y, b0.x, fmaf(-a.x, b0.y, m0i));
            m1r = fmaf(a.x, b1.x, fmaf(a.y, b1.y, m1r));
            m1i = fmaf(a.y, b1.x, fmaf(-a.x, b1.y, m1i));
        }
        s_M[warp][ca_i * NPX + cb_i] = make_float2(m0r, m0i);
        s_M[warp][ca_i * NPX + cb_i + 4] = make_float2(m1r, m1i);
        __syncwarp();
        if (lane < NL) {
            // ACF(ux, uy) = sum_a M[a][a + ux]
            float ar = 0.0f, ai = 0.0f;
#pragma unroll
            for (int a = 0; a < NPX; ++a) {
                int b = a + ux;
                if (b >= 0 && b < NPX) {
                    float2 m = s_M[warp][a * NPX + b];
                    ar += m.x;
                    ai += m.y;
                }
            }
            float otf = 1.0f;
            if (sd.elong_a > 0.0f) {
                float d = (float)ux * sd.dir_x + (float)uy * sd.dir_y;
                otf = expf(-sd.elong_a * d * d);
            }
            float2 hh = cmul(hx, w.h[uy + NPX - 1]);
            float2 p = cmul(make_float2(ar * otf, ai * otf), hh);
            s_P[warp][uy * NL + lane] = p;
        }
        __syncwarp();
    }

    // Y[uy][mx] = sum_ux P(ux, uy) e^{2 pi i ux mx / ND}, uy >= 0
#pragma unroll
    for (int j = 0; j < Y_PER_LANE; ++j) {
        int o = lane + 32 * j;
        if (o < NPX * ND) {
            int uy = o / ND, mx = o % ND;
            const float2* prow = s_P[warp] + uy * NL;
            float yr = 0.0f, yi = 0.0f;
#pragma unroll
            for (int q = 0; q < NL; ++q) {
                int m = (((q - (NPX - 1)) % ND + ND) * mx) % ND;
                float2 t = s_tw[warp][m], p = prow[q];
                yr = fmaf(p.x, t.x, fmaf(-p.y, t.y, yr));
                yi = fmaf(p.x, t.y, fmaf(p.y, t.x, yi));
            }
            s_Y[warp][o] = make_float2(yr, yi);
        }
    }
    __syncwarp();

    // B[my][mx] = Re(Y[0][mx]) + 2 Re sum_{uy>0} Y[uy][mx] e^{2 pi i uy my / ND}
    float B[PIX_PER_LANE];
    float bsum = 0.0f;
#pragma unroll
    for (int j = 0; j < PIX_PER_LANE; ++j) {
        int o = lane + 32 * j;
        float b = 0.0f;
        if (o < ND * ND) {
            int my = o / ND, mx = o % ND;
            float acc = 0.0f;
#pragma unroll
            for (int uy = 1; uy < NPX; ++uy) {
                float2 t = s_tw[warp][(uy * my) % ND], yv = s_Y[warp][uy * ND + mx];
                acc = fmaf(yv.x, t.x, fmaf(-yv.y, t.y, acc));
            }
            b = fmaf(2.0f, acc, s_Y[warp][mx].x);
        }
        B[j] = b;
        bsum += b;
    }
    bsum = warp_sum(bsum);
    const float norm = (bsum > 0.0f) ? w.n_photons * sd.frac / bsum : 0.0f;

    // detector pixels: expected photo-electrons, optional noise, centre of gravity
    const float c0 = 0.5f * (float)(ND - 1);
    float sv = 0.0f, sx = 0.0f, sy = 0.0f;
    const long long pix0 = (long long)sd.rank * ND * ND;
#pragma unroll
    for (int j = 0; j < PIX_PER_LANE; ++j) {
        int o = lane + 32 * j;
        if (o < ND * ND) {
            float lam = B[j] * norm;
            float v = lam;
            if (L.ctx.noise) {
                int n = noise_sample(lam, w.read_noise, (uint32_t)(pix0 + o), (uint32_t)k, (uint32_t)w.wfs_index,
                                     L.ctx.seed, s_recip[warp]);
                v = (float)n;
                if (L.frame_out) L.frame_out[w.frame0 + pix0 + o] = n;
            }
            if (L.lam_out) L.lam_out[w.frame0 + pix0 + o] = lam;
            int my = o / ND, mx = o % ND;
            sv += v;
            sx = fmaf((float)mx - c0, v, sx);
            sy = fmaf((float)my - c0, v, sy);
        }
    }
    sv = warp_sum(sv);
    sx = warp_sum(sx);
    sy = warp_sum(sy);
    if (lane == 0) {
        float gx = 0.0f, gy = 0.0f;
        if (sv > 0.0f) {
            gx = sx / sv;
            gy = sy / sv;
        }
        int ix = w.slope0 + sd.rank, iy = w.slope0 + w.n_valid + sd.rank;
        L.slopes[ix] = gx - (L.s_ref ? L.s_ref[ix] : 0.0f);
        L.slopes[iy] = gy - (L.s_ref ? L.s_ref[iy] : 0.0f);
    }
}

// ------------------------------------------------------------------------------------------
// FFT route: one 1024-thread block per subaperture, no elongation
// ------------------------------------------------------------------------------------------
constexpr int kFftThreads = 1024;

template <int NPX, int NFFT, int NBIN>
__global__ void __launch_bounds__(kFftThreads) wfs_fft_kernel(WfsLaunch L) {
    constexpr int ND = NFFT / NBIN;
    constexpr int NT = kFftThreads;
    constexpr int NW = NT / 32;
    extern __shared__ float4 smem_raw[];
    float2* X = reinterpret_cast<float2*>(smem_raw);              // [NFFT][NFFT]
    float2* Z = X + NFFT * NFFT;                                   // [NFFT][NFFT]
    float2* W = Z + NFFT * NFFT;                                   // [NFFT]
    AxisEnt* ex = reinterpret_cast<AxisEnt*>(W + NFFT);            // [kMaxEntries * NPX]
    AxisEnt* ey = ex + kMaxEntries * NPX;                          // [kMaxEntries * NPX]
    float* recip = reinterpret_cast<float*>(ey + kMaxEntries * NPX);  // [65]
    float* red = recip + 68;                                       // [3 * NW]

    const int tid = threadIdx.x;
    const SubapDev sd = L.subaps[blockIdx.x];
    const WfsDev& w = L.ctx.wfs[sd.wfs];
    const int i0 = sd.sx * NPX, j0 = sd.sy * NPX;
    const int n_grids = L.ctx.n_grids;
    const GridView* V = L.ctx.views + (long long)sd.wfs * n_grids;
    const long long k = L.ctx.st->k;

    tile_entries(V, n_grids, k, i0, j0, NPX, ex, ey, tid, NT);
    if (L.ctx.noise) fill_recip(recip, tid, NT);
    for (int q = tid; q < NFFT; q += NT) {
        float s, c;
        sincospif(-2.0f * (float)q / (float)NFFT, &s, &c);
        W[q] = make_float2(c, s);
    }
    for (int q = tid; q < NFFT * NFFT; q += NT) {
        X[q] = make_float2(0.0f, 0.0f);
        Z[q] = make_float2(0.0f, 0.0f);
    }
    __syncthreads();
    const float scale = w.scale;
    for (int q = tid; q < NPX * NPX; q += NT) {
        int x = q % NPX, y = q / NPX;
        float phi = tile_phase(V, n_grids, ex, ey, NPX, x, y);
        float a = __ldg(w.amp + (long long)(j0 + y) * w.N + i0 + x);
        float arg = scale * phi - kPi * (float)(x + y) / (float)NFFT;
        float sn, cs;
        sincosf(arg, &sn, &cs);
        X[y * NFFT + x] = make_float2(a * cs, a * sn);
    }
    __syncthreads();
    int rad[8];
    int nr = 0;
    for (int n = NFFT; n > 1;) {
        int r = (n % 4 == 0) ? 4 : 2;
        rad[nr++] = r;
        n /= r;
    }
    // rows holding the field (others are zero), then every column
    float2* R1 = stockham_fft(X, Z, NFFT, rad, nr, NPX, NFFT, 1, W, tid, NT);
    float2* R2 = stockham_fft(R1, R1 == X ? Z : X, NFFT, rad, nr, NFFT, 1, NFFT, W, tid, NT);

    // |.|^2, shift by NFFT/2, bin NBIN x NBIN
    const int lane = tid & 31, warp = tid >> 5;
    float b = 0.0f;
    const int o = tid;
    const int my = o / ND, mx = o % ND;
    if (o < ND * ND) {
        for (int ty = 0; ty < NBIN; ++ty)
            for (int tx = 0; tx < NBIN; ++tx) {
                int r = (my * NBIN + ty + NFFT / 2) % NFFT, c = (mx * NBIN + tx + NFFT / 2) % NFFT;
                float2 v = R2[r * NFFT + c];
                b += v.x * v.x + v.y * v.y;
            }
    }
    float s = warp_sum(b);
    if (lane == 0) red[warp] = s;
    __syncthreads();
    float bsum = 0.0f;
    for (int q = 0; q < NW; ++q) bsum += red[q];
    const float norm = (bsum > 0.0f) ? w.n_photons * sd.frac / bsum : 0.0f;
    __syncthreads();

    const float c0 = 0.5f * (float)(ND - 1);
    float sv = 0.0f, sx = 0.0f, sy = 0.0f;
    const long long pix0 = (long long)sd.rank * ND * ND;
    if (o < ND * ND) {
        float lam = b * norm;
        float v = lam;
        if (L.ctx.noise) {
            int n = noise_sample(lam, w.read_noise, (uint32_t)(pix0 + o), (uint32_t)k, (uint32_t)w.wfs_index,
                                 L.ctx.seed, recip);
            v = (float)n;
            if (L.frame_out) L.frame_out[w.frame0 + pix0 + o] = n;
        }
        if (L.lam_out) L.lam_out[w.frame0 + pix0 + o] = lam;
        sv = v;
        sx = ((float)mx - c0) * v;
        sy = ((float)my - c0) * v;
    }
    sv = warp_sum(sv);
    sx = warp_sum(sx);
    sy = warp_sum(sy);
    if (lane == 0) {
        red[warp] = sv;
        red[NW + warp] = sx;
        red[2 * NW + warp] = sy;
    }
    __syncthreads();
    if (tid == 0) {
        float tv = 0.0f, tx = 0.0f, ty = 0.0f;
        for (int q = 0; q < NW; ++q) {
            tv += red[q];
            tx += red[NW + q];
            ty += red[2 * NW + q];
        }
        float gx = 0.0f, gy = 0.0f;
        if (tv > 0.0f) {
            gx = tx / tv;
            gy = ty / tv;
        }
        int ix = w.slope0 + sd.rank, iy = w.slope0 + w.n_valid + sd.rank;
        L.slopes[ix] = gx - (L.s_ref ? L.s_ref[ix] : 0.0f);
        L.slopes[iy] = gy - (L.s_ref ? L.s_ref[iy] : 0.0f);
    }
}

template <int NPX, int NFFT>
constexpr size_t fft_smem() {
    return sizeof(float2) * (2 * NFFT * NFFT + NFFT) + sizeof(AxisEnt) * 2 * kMaxEntries * NPX +
           sizeof(float) * (68 + 3 * (kFftThreads / 32));
}

// residual phase on the full pupil grid of one WFS, 8 x 8 tiles, one warp per tile
__global__ void __launch_bounds__(256) wfs_phase_kernel(Ctx ctx, int wi, int N, float* out) {
    __shared__ AxisEnt s_ex[8][kMaxEntries * 8];
    __shared__ AxisEnt s_ey[8][kMaxEntries * 8];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int tiles_x = (N + 7) / 8;
    const int tile = blockIdx.x * 8 + warp;
    if (tile >= tiles_x * tiles_x) return;
    const int i0 = (tile % tiles_x) * 8, j0 = (tile / tiles_x) * 8;
    const GridView* V = ctx.views + (long long)wi * ctx.n_grids;
    tile_entries(V, ctx.n_grids, ctx.st->k, i0, j0, 8, s_ex[warp], s_ey[warp], lane, 32);
    __syncwarp();
    for (int q = lane; q < 64; q += 32) {
        int x = q % 8, y = q / 8;
        if (i0 + x < N && j0 + y < N)
            out[(long long)(j0 + y) * N + i0 + x] = tile_phase(V, ctx.n_grids, s_ex[warp], s_ey[warp], 8, x, y);
    }
}

template <int NFFT, int NBIN>
cudaError_t launch_acf(const WfsLaunch& L, cudaStream_t s) {
    unsigned blocks = (unsigned)((L.n_subaps + 7) / 8);
    if (blocks) wfs_acf_kernel<NFFT, NBIN><<<blocks, 256, 0, s>>>(L);
    return cudaGetLastError();
}

template <int NPX, int NFFT, int NBIN>
cudaError_t prepare_fft() {
    return cudaFuncSetAttribute(wfs_fft_kernel<NPX, NFFT, NBIN>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                (int)fft_smem<NPX, NFFT>());
}

template <int NPX, int NFFT, int NBIN>
cudaError_t launch_fft(const WfsLaunch& L, cudaStream_t s) {
    constexpr size_t sm = fft_smem<NPX, NFFT>();
    if (L.n_subaps) wfs_fft_kernel<NPX, NFFT, NBIN><<<(unsigned)L.n_subaps, kFftThreads, sm, s>>>(L);
    return cudaGetLastError();
}

}  // namespace

bool wfs_variant_supported(int n_px, int n_fft, int n_bin, bool elongated) {
    if (n_px == 8 && n_fft == 16 && n_bin == 2) return true;
    if (n_px == 8 && n_fft == 32 && n_bin == 2) return true;
    if (n_px == 8 && n_fft == 16 && n_bin == 1) return true;
    if (n_px == 32 && n_fft == 64 && n_bin == 4) return !elongated;
    return false;
}

bool wfs_variant_is_fft(int n_px, int n_fft, int n_bin) { return n_px == 32 && n_fft == 64 && n_bin == 4; }

cudaError_t wfs_prepare() { return prepare_fft<32, 64, 4>(); }

cudaError_t launch_wfs(const WfsLaunch& L, int n_px, int n_fft, int n_bin, cudaStream_t s) {
    if (n_px == 8 && n_fft == 16 && n_bin == 2) return launch_acf<16, 2>(L, s);
    if (n_px == 8 && n_fft == 32 && n_bin == 2) return launch_acf<32, 2>(L, s);
    if (n_px == 8 && n_fft == 16 && n_bin == 1) return launch_acf<16, 1>(L, s);
    if (n_px == 32 && n_fft == 64 && n_bin == 4) return launch_fft<32, 64, 4>(L, s);
    return cudaErrorInvalidValue;
}

cudaError_t launch_wfs_phase(const Ctx& ctx, int wfs, int N, float* out, cudaStream_t s) {
    int tiles = ((N + 7) / 8) * ((N + 7) / 8);
    wfs_phase_kernel<<<(unsigned)((tiles + 7) / 8), 256, 0, s>>>(ctx, wfs, N, out);
    return cudaGetLastError();
}

}  // namespace mcao
