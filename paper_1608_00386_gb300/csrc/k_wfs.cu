// Shack-Hartmann wavefront sensing of the residual phase ("The closed loop" of
// arXiv:1608.00386: the WFS modules compute X and Y slopes from the open-loop wavefront minus
// the DMs), fused per subaperture: cone-beam propagation of every layer and DM, field
// A exp(i phi), spot formation, sodium elongation, binning, flux normalisation, photon and read
// noise, centre of gravity minus the reference slopes.
//
// Spot formation.  The defining computation is: zero-pad the n x n field to N x N, I = |FFT2|^2,
// elongate by FFT2(I) * OTF -> IFFT2, fftshift, bin b x b.  Two kernels compute exactly that
// result by cheaper routes:
//  * autocorrelation route (small subapertures, with or without elongation): FFT2(I)(u) equals
//    N^2 sum_y E(y - u) conj(E(y)), nonzero only for |u| <= n-1 < N/2.  Shift by N/2 and
//    b x b binning are, in the frequency domain, the factor h(u) = (-1)^u sum_{t<b} e^{2 pi i u t/N}
//    per axis followed by an (N/b)-point inverse DFT of the lags, so the detector frame is
//    B[m] = sum_u ACF(u) OTF(u) h(ux) h(uy) e^{2 pi i u.m / n_det} (up to a constant that the
//    flux normalisation removes).  One warp per subaperture; no N x N array is formed.
//  * FFT route (large subapertures without elongation, e.g. 2 x 2 low-order sensors):
//    radix-4 Stockham FFTs of the padded field in shared memory, |.|^2, shift and bin.
#include <math.h>

#include "device_common.cuh"
#include "mcao_internal.h"

namespace mcao {

namespace {

constexpr float kPi = 3.14159265358979323846f;

// coefficients of every grid for a tile, computed by threads [0, n_grids)
__device__ __forceinline__ void tile_coefs(const Ctx& ctx, const WfsDev& w, int i0, int j0, Coef* out,
                                           int tid) {
    if (tid < ctx.n_grids) {
        double t = (double)ctx.st->k * ctx.dt;
        double H = (w.type == 1) ? w.height : 0.0;
        out[tid] = make_coef(ctx.grids[tid], (double)w.N, w.dx, w.theta_x, w.theta_y, H, t, i0, j0);
    }
}

__device__ __forceinline__ float tile_phase(const Coef* cf, int n_grids, float x, float y) {
    float phi = 0.0f;
    for (int g = 0; g < n_grids; ++g) phi += sample_coef(cf[g], x, y);
    return phi;
}

// ------------------------------------------------------------------------------------------
// autocorrelation route: one warp per subaperture, 8 warps per block
// ------------------------------------------------------------------------------------------
template <int NPX, int NFFT, int NBIN>
__global__ void __launch_bounds__(256) wfs_acf_kernel(WfsLaunch L) {
    constexpr int ND = NFFT / NBIN;
    constexpr int NL = 2 * NPX - 1;
    constexpr int NP = NPX * NPX;
    constexpr int NH = NPX * NL - (NPX - 1);  // half-plane lags
    constexpr int PIX_PER_LANE = (ND * ND + 31) / 32;
    __shared__ Coef s_cf[8][kMaxEntries];
    __shared__ float2 s_E[8][NP];
    __shared__ float2 s_P[8][NL * NL];
    __shared__ float2 s_Y[8][NPX * ND];

    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int sub = blockIdx.x * 8 + warp;
    if (sub >= L.n_subaps) return;  // warp-uniform; the kernel uses warp-level sync only
    const SubapDev sd = L.subaps[sub];
    const WfsDev& w = L.ctx.wfs[sd.wfs];
    const int i0 = sd.sx * NPX, j0 = sd.sy * NPX;
    Coef* cf = s_cf[warp];
    float2* E = s_E[warp];
    float2* P = s_P[warp];
    float2* Y = s_Y[warp];

    tile_coefs(L.ctx, w, i0, j0, cf, lane);
    __syncwarp();

    // field E = A exp(i (scale phi - pi (x + y) / N)), half-bin centring ramp
    const float scale = w.scale;
    for (int q = lane; q < NP; q += 32) {
        int x = q % NPX, y = q / NPX;
        float phi = tile_phase(cf, L.ctx.n_grids, (float)x, (float)y);
        float a = __ldg(w.amp + (long long)(j0 + y) * w.N + i0 + x);
        float arg = scale * phi - kPi * (float)(x + y) / (float)NFFT;
        float sn, cs;
        sincosf(arg, &sn, &cs);
        E[q] = make_float2(a * cs, a * sn);
    }
    __syncwarp();

    // lags u = (ux, uy), uy >= 0 half plane: P(u) = ACF(u) OTF(u) h(ux) h(uy); P(-u) = conj P(u)
    for (int hq = lane; hq < NH; hq += 32) {
        int qf = hq + (NPX - 1);
        int uy = qf / NL, ux = qf % NL - (NPX - 1);
        float ar = 0.0f, ai = 0.0f;
        int x_lo = ux > 0 ? ux : 0, x_hi = ux < 0 ? NPX + ux : NPX;
        for (int yy = uy; yy < NPX; ++yy) {
            const int r1 = (yy - uy) * NPX - ux, r2 = yy * NPX;  // E(y - u), E(y)
            for (int yx = x_lo; yx < x_hi; ++yx) {
                float2 a = E[r1 + yx], b = E[r2 + yx];
                ar = fmaf(a.x, b.x, fmaf(a.y, b.y, ar));   // a conj(b)
                ai = fmaf(a.y, b.x, fmaf(-a.x, b.y, ai));
            }
        }
        float otf = 1.0f;
        if (sd.elong_a > 0.0f) {
            float d = (float)ux * sd.dir_x + (float)uy * sd.dir_y;
            otf = expf(-sd.elong_a * d * d);
        }
        float2 hx = w.h[ux + NPX - 1], hy = w.h[uy + NPX - 1];
        float2 hh = cmul(hx, hy);
        float2 p = make_float2(ar * otf, ai * otf);
        p = cmul(p, hh);
        P[(uy + NPX - 1) * NL + (ux + NPX - 1)] = p;
        P[(-uy + NPX - 1) * NL + (-ux + NPX - 1)] = make_float2(p.x, -p.y);
    }
    __syncwarp();

    // Y[uy][mx] = sum_ux P(ux, uy) e^{2 pi i ux mx / ND}, uy >= 0
    for (int o = lane; o < NPX * ND; o += 32) {
        int uy = o / ND, mx = o % ND;
        const float2* prow = P + (uy + NPX - 1) * NL;
        float yr = 0.0f, yi = 0.0f;
#pragma unroll
        for (int ux = -(NPX - 1); ux < NPX; ++ux) {
            int m = ((ux % ND + ND) * mx) % ND;
            float2 t = w.tw[m], p = prow[ux + NPX - 1];
            yr = fmaf(p.x, t.x, fmaf(-p.y, t.y, yr));
            yi = fmaf(p.x, t.y, fmaf(p.y, t.x, yi));
        }
        Y[o] = make_float2(yr, yi);
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
                float2 t = w.tw[(uy * my) % ND], yv = Y[uy * ND + mx];
                acc = fmaf(yv.x, t.x, fmaf(-yv.y, t.y, acc));
            }
            b = fmaf(2.0f, acc, Y[mx].x);
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
    const unsigned k = (unsigned)L.ctx.st->k;
#pragma unroll
    for (int j = 0; j < PIX_PER_LANE; ++j) {
        int o = lane + 32 * j;
        if (o < ND * ND) {
            float lam = B[j] * norm;
            float v = lam;
            if (L.ctx.noise) {
                int n = noise_sample(lam, w.read_noise, (uint32_t)(pix0 + o), k, (uint32_t)w.wfs_index,
                                     L.ctx.seed);
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
// FFT route: one block (256 threads) per subaperture, no elongation
// ------------------------------------------------------------------------------------------
template <int NPX, int NFFT, int NBIN>
__global__ void __launch_bounds__(256) wfs_fft_kernel(WfsLaunch L) {
    constexpr int ND = NFFT / NBIN;
    constexpr int NT = 256;
    extern __shared__ float4 smem_raw[];
    float2* X = reinterpret_cast<float2*>(smem_raw);          // [NFFT][NFFT]
    float2* Z = X + NFFT * NFFT;                               // [NFFT][NFFT]
    float2* W = Z + NFFT * NFFT;                               // [NFFT]
    Coef* cf = reinterpret_cast<Coef*>(W + NFFT);              // [kMaxEntries]
    float* red = reinterpret_cast<float*>(cf + kMaxEntries);   // [3 * 8]

    const int tid = threadIdx.x;
    const SubapDev sd = L.subaps[blockIdx.x];
    const WfsDev& w = L.ctx.wfs[sd.wfs];
    const int i0 = sd.sx * NPX, j0 = sd.sy * NPX;

    tile_coefs(L.ctx, w, i0, j0, cf, tid);
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
        float phi = tile_phase(cf, L.ctx.n_grids, (float)x, (float)y);
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
    float lam = 0.0f, b = 0.0f;
    int o = tid;
    int my = o / ND, mx = o % ND;
    if (o < ND * ND) {
        for (int ty = 0; ty < NBIN; ++ty)
            for (int tx = 0; tx < NBIN; ++tx) {
                int r = (my * NBIN + ty + NFFT / 2) % NFFT, c = (mx * NBIN + tx + NFFT / 2) % NFFT;
                float2 v = R2[r * NFFT + c];
                b += v.x * v.x + v.y * v.y;
            }
    }
    const int lane = tid & 31, warp = tid >> 5;
    float s = warp_sum(b);
    if (lane == 0) red[warp] = s;
    __syncthreads();
    float bsum = 0.0f;
    for (int q = 0; q < NT / 32; ++q) bsum += red[q];
    const float norm = (bsum > 0.0f) ? w.n_photons * sd.frac / bsum : 0.0f;
    __syncthreads();

    const float c0 = 0.5f * (float)(ND - 1);
    float sv = 0.0f, sx = 0.0f, sy = 0.0f;
    const long long pix0 = (long long)sd.rank * ND * ND;
    if (o < ND * ND) {
        lam = b * norm;
        float v = lam;
        if (L.ctx.noise) {
            int n = noise_sample(lam, w.read_noise, (uint32_t)(pix0 + o), (unsigned)L.ctx.st->k,
                                 (uint32_t)w.wfs_index, L.ctx.seed);
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
        red[8 + warp] = sx;
        red[16 + warp] = sy;
    }
    __syncthreads();
    if (tid == 0) {
        float tv = 0.0f, tx = 0.0f, ty = 0.0f;
        for (int q = 0; q < NT / 32; ++q) {
            tv += red[q];
            tx += red[8 + q];
            ty += red[16 + q];
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

template <int NFFT>
constexpr size_t fft_smem() {
    return sizeof(float2) * (2 * NFFT * NFFT + NFFT) + sizeof(Coef) * kMaxEntries + sizeof(float) * 24;
}

// residual phase on the full pupil grid of one WFS, 8 x 8 tiles, one warp per tile
__global__ void __launch_bounds__(256) wfs_phase_kernel(Ctx ctx, int wi, int N, float* out) {
    __shared__ Coef s_cf[8][kMaxEntries];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int tiles_x = (N + 7) / 8;
    const int tile = blockIdx.x * 8 + warp;
    if (tile >= tiles_x * tiles_x) return;
    const WfsDev& w = ctx.wfs[wi];
    const int i0 = (tile % tiles_x) * 8, j0 = (tile / tiles_x) * 8;
    tile_coefs(ctx, w, i0, j0, s_cf[warp], lane);
    __syncwarp();
    for (int q = lane; q < 64; q += 32) {
        int x = q % 8, y = q / 8;
        if (i0 + x < N && j0 + y < N)
            out[(long long)(j0 + y) * N + i0 + x] = tile_phase(s_cf[warp], ctx.n_grids, (float)x, (float)y);
    }
}

template <int NPX, int NFFT, int NBIN>
cudaError_t launch_acf(const WfsLaunch& L, cudaStream_t s) {
    unsigned blocks = (unsigned)((L.n_subaps + 7) / 8);
    if (blocks) wfs_acf_kernel<NPX, NFFT, NBIN><<<blocks, 256, 0, s>>>(L);
    return cudaGetLastError();
}

template <int NPX, int NFFT, int NBIN>
cudaError_t prepare_fft() {
    return cudaFuncSetAttribute(wfs_fft_kernel<NPX, NFFT, NBIN>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                (int)fft_smem<NFFT>());
}

template <int NPX, int NFFT, int NBIN>
cudaError_t launch_fft(const WfsLaunch& L, cudaStream_t s) {
    constexpr size_t sm = fft_smem<NFFT>();
    if (L.n_subaps) wfs_fft_kernel<NPX, NFFT, NBIN><<<(unsigned)L.n_subaps, 256, sm, s>>>(L);
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

cudaError_t wfs_prepare() { return prepare_fft<32, 64, 4>(); }

cudaError_t launch_wfs(const WfsLaunch& L, int n_px, int n_fft, int n_bin, cudaStream_t s) {
    if (n_px == 8 && n_fft == 16 && n_bin == 2) return launch_acf<8, 16, 2>(L, s);
    if (n_px == 8 && n_fft == 32 && n_bin == 2) return launch_acf<8, 32, 2>(L, s);
    if (n_px == 8 && n_fft == 16 && n_bin == 1) return launch_acf<8, 16, 1>(L, s);
    if (n_px == 32 && n_fft == 64 && n_bin == 4) return launch_fft<32, 64, 4>(L, s);
    return cudaErrorInvalidValue;
}

cudaError_t launch_wfs_phase(const Ctx& ctx, int wfs, int N, float* out, cudaStream_t s) {
    int tiles = ((N + 7) / 8) * ((N + 7) / 8);
    wfs_phase_kernel<<<(unsigned)((tiles + 7) / 8), 256, 0, s>>>(ctx, wfs, N, out);
    return cudaGetLastError();
}

}  // namespace mcao
