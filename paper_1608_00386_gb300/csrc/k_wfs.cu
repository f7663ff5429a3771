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
//  * FFT route (larger subapertures: 2 x 2 low-order sensors, laser stars with 16 samples per
//    subaperture for a wider field): radix-4 Stockham FFTs of the padded field in shared
//    memory, |.|^2, elongation by two more 2-D FFTs and the OTF, shift and bin; one 1024-thread
//    block per subaperture.
#include <math.h>

#include "device_common.cuh"
#include "mcao_internal.h"

namespace mcao {

namespace {

constexpr float kPi = 3.14159265358979323846f;

// ------------------------------------------------------------------------------------------
// small inverse DFTs in registers: out[k] = sum_j in[j] exp(+2 pi i j k / M), M = 1, 2, 4, 8
// ------------------------------------------------------------------------------------------
template <int M>
__device__ __forceinline__ void idft_small(float2* v);

template <>
__device__ __forceinline__ void idft_small<1>(float2*) {}

template <>
__device__ __forceinline__ void idft_small<2>(float2* v) {
    float2 a = v[0], b = v[1];
    v[0] = cadd(a, b);
    v[1] = csub(a, b);
}

template <>
__device__ __forceinline__ void idft_small<4>(float2* v) {
    float2 a0 = cadd(v[0], v[2]), a1 = csub(v[0], v[2]);
    float2 a2 = cadd(v[1], v[3]), d = csub(v[1], v[3]);
    float2 a3 = make_float2(-d.y, d.x);  // +i (v1 - v3)
    v[0] = cadd(a0, a2);
    v[2] = csub(a0, a2);
    v[1] = cadd(a1, a3);
    v[3] = csub(a1, a3);
}

template <>
__device__ __forceinline__ void idft_small<8>(float2* v) {
    // radix-2 split: even / odd 4-point transforms, twiddles exp(+2 pi i k / 8)
    float2 e[4] = {v[0], v[2], v[4], v[6]}, o[4] = {v[1], v[3], v[5], v[7]};
    idft_small<4>(e);
    idft_small<4>(o);
    const float r = 0.707106781186547524f;
    float2 t1 = make_float2(r * (o[1].x - o[1].y), r * (o[1].x + o[1].y));    // o1 (1 + i)/sqrt2
    float2 t2 = make_float2(-o[2].y, o[2].x);                                 // o2 i
    float2 t3 = make_float2(-r * (o[3].x + o[3].y), r * (o[3].x - o[3].y));   // o3 (-1 + i)/sqrt2
    v[0] = cadd(e[0], o[0]);
    v[4] = csub(e[0], o[0]);
    v[1] = cadd(e[1], t1);
    v[5] = csub(e[1], t1);
    v[2] = cadd(e[2], t2);
    v[6] = csub(e[2], t2);
    v[3] = cadd(e[3], t3);
    v[7] = csub(e[3], t3);
}

// ------------------------------------------------------------------------------------------
// autocorrelation route: one warp per 8 x 8 subaperture, 8 warps per block
// ------------------------------------------------------------------------------------------
struct GridMeta {
    const float* data;
    int n;
    float sign;
};

template <int NFFT, int NBIN>
__global__ void __launch_bounds__(256, 4) wfs_acf_kernel(WfsLaunch L) {
    constexpr int NPX = 8;
    constexpr int ND = NFFT / NBIN;
    constexpr int NL = 2 * NPX - 1;
    constexpr int PIX_PER_LANE = ND * ND / 32;
    constexpr int QY = ND / 4;        // outputs per lane of the row transform (4 lanes per row)
    constexpr int LPC = 32 / ND;      // lanes per column of the column transform
    constexpr int QB = ND / LPC;      // outputs per lane of the column transform
    static_assert(ND == 8 || ND == 16, "detector of 8 or 16 pixels per side");
    // per warp: axis entries (dead after the field, then reused for the second lag row of each
    // pass and for the row transform),
    // grid metadata, the field (reused for M_uy), the lag products; per block: twiddles and
    // reciprocals.  About 30 KB per block, so three blocks fit beside a reconstructor block.
    union Scratch {
        AxisEnt e[2][kMaxEntries * NPX];
        float2 y[NPX * ND];
    };
    static_assert(sizeof(Scratch) >= NPX * NPX * sizeof(float2), "room for one lag row's M");
    __shared__ Scratch s_u[8];
    __shared__ GridMeta s_gm[8][kMaxEntries];
    __shared__ float2 s_EM[8][NPX * NPX];
    __shared__ float2 s_P[8][NPX * NL];
    __shared__ float2 s_tw[ND];
    __shared__ float s_recip[kRecipEntries];

    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    if (threadIdx.x < ND) {
        float sn, cs;
        sincospif(2.0f * (float)threadIdx.x / (float)ND, &sn, &cs);  // exp(2 pi i k / ND)
        s_tw[threadIdx.x] = make_float2(cs, sn);
    }
    if (L.ctx.noise) fill_recip(s_recip, threadIdx.x, blockDim.x);
    __syncthreads();  // the only block-wide barrier
    // subapertures: one per warp (no counter), or taken one at a time from the counter, so that
    // warps of blocks that become resident late take only what is left
    auto take = [&]() {
        unsigned int v = 0;
        if (lane == 0) v = atomicAdd(L.work, 1u);
        return (int)__shfl_sync(0xffffffffu, v, 0);
    };
    // items run over (realization, subaperture)
    const int n_items = L.n_subaps * L.ctx.n_real;
    int item = L.work ? take() : blockIdx.x * 8 + warp;
    for (;;) {
        if (item >= n_items) break;  // warp-uniform; warp-level sync only from here on
        const int real = item / L.n_subaps, sub = item - real * L.n_subaps;
        const SubapDev sd = L.subaps[sub];
        const WfsDev& w = L.ctx.wfs[sd.wfs];
        const int i0 = sd.sx * NPX, j0 = sd.sy * NPX;
        const int n_grids = L.ctx.n_grids;
        const GridView* V = L.ctx.views + real * L.ctx.view_stride + (long long)sd.wfs * n_grids;
        const long long k = L.ctx.st->k;
        AxisEnt* s_ex = s_u[warp].e[0];
        AxisEnt* s_ey = s_u[warp].e[1];

        tile_entries<NPX>(V, n_grids, k, i0, j0, s_ex, s_ey, lane, 32);
        if (lane < n_grids) {
            GridMeta gm;
            gm.data = V[lane].data;
            gm.n = V[lane].n;
            gm.sign = V[lane].sign;
            s_gm[warp][lane] = gm;
        }
        __syncwarp();

        // field E = A exp(i (scale phi - pi (x + y) / N)): lane -> column x, rows y0 and y0 + 4
        {
            const int x = lane & 7, y0 = lane >> 3, y1 = y0 + 4;
            float phi0 = 0.0f, phi1 = 0.0f;
    #pragma unroll 2
            for (int g = 0; g < n_grids; ++g) {
                const GridMeta gm = s_gm[warp][g];
                const AxisEnt ex = s_ex[g * NPX + x];
                phi0 = fmaf(gm.sign, bilinear(gm.data, gm.n, ex, s_ey[g * NPX + y0]), phi0);
                phi1 = fmaf(gm.sign, bilinear(gm.data, gm.n, ex, s_ey[g * NPX + y1]), phi1);
            }
            const float scale = w.scale;
            const float* arow = w.amp + (long long)j0 * w.N + i0 + x;
            float a0 = __ldg(arow + (long long)y0 * w.N), a1 = __ldg(arow + (long long)y1 * w.N);
            float sn, cs;
            sincosf(scale * phi0 - kPi * (float)(x + y0) / (float)NFFT, &sn, &cs);
            s_EM[warp][y0 * NPX + x] = make_float2(a0 * cs, a0 * sn);
            sincosf(scale * phi1 - kPi * (float)(x + y1) / (float)NFFT, &sn, &cs);
            s_EM[warp][y1 * NPX + x] = make_float2(a1 * cs, a1 * sn);
        }
        __syncwarp();

        // ACF(ux, uy) = sum_a M_uy[a][a + ux], M_uy[a][b] = sum_r E[r][a] conj(E[r + uy][b]);
        // lane holds columns a, b0, b1 of E
        {
            const int ca_i = lane >> 2, cb_i = lane & 3;
            float2 ca[NPX], cb0[NPX], cb1[NPX];
    #pragma unroll
            for (int r = 0; r < NPX; ++r) {
                ca[r] = s_EM[warp][r * NPX + ca_i];
                cb0[r] = s_EM[warp][r * NPX + cb_i];
                cb1[r] = s_EM[warp][r * NPX + cb_i + 4];
            }
            __syncwarp();  // every lane holds its columns: the buffers now receive M_uy
            // two lag rows per pass: M_uy in the field's buffer, M_{uy+1} in this warp's axis-entry
            // scratch (dead after the field); lanes 0..14 sum the diagonals of row uy, lanes
            // 16..30 those of row uy + 1 (ux = (lane mod 16) - 7)
            float2* s_M1 = reinterpret_cast<float2*>(&s_u[warp]);
            const int half = lane >> 4, uxl = lane & 15;
            const bool diag = uxl < NL;
            const int ux = uxl - (NPX - 1);
            float2 hx = make_float2(0.0f, 0.0f);
            if (diag) hx = w.h[uxl];  // h(ux)
    #pragma unroll
            for (int uy0 = 0; uy0 < NPX; uy0 += 2) {
                float m0r = 0.0f, m0i = 0.0f, m1r = 0.0f, m1i = 0.0f;
                float n0r = 0.0f, n0i = 0.0f, n1r = 0.0f, n1i = 0.0f;
    #pragma unroll
                for (int r = 0; r + uy0 < NPX; ++r) {
                    float2 a = ca[r], b0 = cb0[r + uy0], b1 = cb1[r + uy0];
                    m0r = fmaf(a.x, b0.x, fmaf(a.y, b0.y, m0r));
                    m0i = fmaf(a.y, b0.x, fmaf(-a.x, b0.y, m0i));
                    m1r = fmaf(a.x, b1.x, fmaf(a.y, b1.y, m1r));
                    m1i = fmaf(a.y, b1.x, fmaf(-a.x, b1.y, m1i));
                }
    #pragma unroll
                for (int r = 0; r + uy0 + 1 < NPX; ++r) {
                    float2 a = ca[r], b0 = cb0[r + uy0 + 1], b1 = cb1[r + uy0 + 1];
                    n0r = fmaf(a.x, b0.x, fmaf(a.y, b0.y, n0r));
                    n0i = fmaf(a.y, b0.x, fmaf(-a.x, b0.y, n0i));
                    n1r = fmaf(a.x, b1.x, fmaf(a.y, b1.y, n1r));
                    n1i = fmaf(a.y, b1.x, fmaf(-a.x, b1.y, n1i));
                }
                s_EM[warp][ca_i * NPX + cb_i] = make_float2(m0r, m0i);
                s_EM[warp][ca_i * NPX + cb_i + 4] = make_float2(m1r, m1i);
                s_M1[ca_i * NPX + cb_i] = make_float2(n0r, n0i);
                s_M1[ca_i * NPX + cb_i + 4] = make_float2(n1r, n1i);
                __syncwarp();
                if (diag) {
                    const float2* M = half ? s_M1 : s_EM[warp];
                    const int uy = uy0 + half;
                    float ar = 0.0f, ai = 0.0f;
    #pragma unroll
                    for (int a = 0; a < NPX; ++a) {
                        int b = a + ux;
                        if (b >= 0 && b < NPX) {
                            float2 m = M[a * NPX + b];
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
                    s_P[warp][uy * NL + uxl] = cmul(make_float2(ar * otf, ai * otf), hh);
                }
                __syncwarp();
            }
        }

        // rows: Y[uy][q + 4 j] = sum_ux P[uy][ux] w^{ux q} (w^4)^{ux j}, w = e^{2 pi i / ND};
        // lane -> (uy, q), fold ux mod ND/4, then an ND/4-point inverse DFT
        {
            const int uy = lane >> 2, q = lane & 3;
            float2 S[QY];
    #pragma unroll
            for (int r = 0; r < QY; ++r) S[r] = make_float2(0.0f, 0.0f);
    #pragma unroll
            for (int c = 0; c < NL; ++c) {
                const int ux = c - (NPX - 1);
                const float2 p = s_P[warp][uy * NL + c];
                const float2 t = s_tw[((ux + 2 * ND) * q) % ND];
                const int r = (ux + 2 * ND) % QY;
                S[r] = cadd(S[r], cmul(p, t));
            }
            idft_small<QY>(S);
    #pragma unroll
            for (int j = 0; j < QY; ++j) s_u[warp].y[uy * ND + q + 4 * j] = S[j];
        }
        __syncwarp();

        // columns: B[h + LPC j][mx] = Re sum_uy z[uy] w^{uy h} (w^LPC)^{uy j}, z = Y[0], 2 Y[uy > 0];
        // lane -> (mx, h); fold uy mod QB, then a QB-point inverse DFT (real part).  Output j of
        // lane l is detector pixel o = l + 32 j.
        float B[PIX_PER_LANE];
        float bsum = 0.0f;
        {
            const int mx = lane & (ND - 1), h = lane / ND;
            static_assert(PIX_PER_LANE == QB, "pixel mapping");
            float2 Z[QB];
    #pragma unroll
            for (int r = 0; r < QB; ++r) Z[r] = make_float2(0.0f, 0.0f);
    #pragma unroll
            for (int uy = 0; uy < NPX; ++uy) {
                float2 y = s_u[warp].y[uy * ND + mx];
                if (uy > 0) y = make_float2(2.0f * y.x, 2.0f * y.y);
                const float2 t = s_tw[(uy * h) % ND];
                Z[uy % QB] = cadd(Z[uy % QB], cmul(y, t));
            }
            idft_small<QB>(Z);
    #pragma unroll
            for (int j = 0; j < QB; ++j) {
                B[j] = Z[j].x;
                bsum += Z[j].x;
            }
        }
        bsum = warp_sum(bsum);
        const float norm = (bsum > 0.0f) ? w.n_photons * sd.frac / bsum : 0.0f;

        // detector pixels o = lane + 32 j = my ND + mx: expected photo-electrons, optional noise,
        // centre of gravity
        const float c0 = 0.5f * (float)(ND - 1);
        float sv = 0.0f, sx = 0.0f, sy = 0.0f;
        const long long pix0 = (long long)sd.rank * ND * ND;
        // pixel pairs (o, o + ND^2 / 2) sit in this lane's slots j and j + PIX_PER_LANE / 2
        constexpr int HALF = PIX_PER_LANE / 2;
    #pragma unroll
        for (int j = 0; j < HALF; ++j) {
            const int o = lane + 32 * j;
            const float lam_a = B[j] * norm, lam_b = B[j + HALF] * norm;
            float va = lam_a, vb = lam_b;
            if (L.ctx.noise) {
                int na, nb;
                noise_pair(lam_a, lam_b, w.read_noise, (uint32_t)(pix0 + o), (uint32_t)k, (uint32_t)w.wfs_index,
                           L.ctx.seed + real, s_recip, na, nb);
                va = (float)na;
                vb = (float)nb;
                if (L.frame_out) {
                    L.frame_out[real * L.frame_stride + w.frame0 + pix0 + o] = na;
                    L.frame_out[real * L.frame_stride + w.frame0 + pix0 + o + 32 * HALF] = nb;
                }
            }
            if (L.lam_out) {
                L.lam_out[real * L.frame_stride + w.frame0 + pix0 + o] = lam_a;
                L.lam_out[real * L.frame_stride + w.frame0 + pix0 + o + 32 * HALF] = lam_b;
            }
            const int my = o / ND, mx = o % ND, my_b = (o + 32 * HALF) / ND;
            sv += va + vb;
            sx = fmaf((float)mx - c0, va + vb, sx);
            sy = fmaf((float)my - c0, va, sy);
            sy = fmaf((float)my_b - c0, vb, sy);
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
            const float vx = gx - (L.s_ref ? L.s_ref[ix] : 0.0f), vy = gy - (L.s_ref ? L.s_ref[iy] : 0.0f);
            float* slopes = L.slopes + (long long)real * L.slope_stride;
            slopes[ix] = vx;
            slopes[iy] = vy;
            if (L.slopes_pad) {
                float* pad = L.slopes_pad + (long long)real * L.pad_stride;
                pad[w.rcol0 + sd.rank] = vx;
                pad[w.rcol0 + w.n_valid + sd.rank] = vy;
            }
        }
        if (!L.work) break;
        item = take();
        __syncwarp();  // the scratch of this subaperture is read before the next one writes it
    }
}

// ------------------------------------------------------------------------------------------
// FFT route: one 1024-thread block per subaperture
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
    float* recip = reinterpret_cast<float*>(ey + kMaxEntries * NPX);  // [kRecipEntries]
    float* red = recip + 68;                                       // [3 * NW]

    const int tid = threadIdx.x;
    const int real = blockIdx.x / L.n_subaps;   // blocks run over (realization, subaperture)
    const SubapDev sd = L.subaps[blockIdx.x - real * L.n_subaps];
    const WfsDev& w = L.ctx.wfs[sd.wfs];
    const int i0 = sd.sx * NPX, j0 = sd.sy * NPX;
    const int n_grids = L.ctx.n_grids;
    const GridView* V = L.ctx.views + real * L.ctx.view_stride + (long long)sd.wfs * n_grids;
    const long long k = L.ctx.st->k;

    tile_entries<NPX>(V, n_grids, k, i0, j0, ex, ey, tid, NT);
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

    // sodium elongation (block-uniform branch): I <- Re IFFT2(FFT2(I) OTF), the inverse taken as
    // conj(FFT2(conj .)) and its 1 / N^2 left to the flux normalisation
    const float2* img = R2;
    const bool elong = sd.elong_a > 0.0f;
    if (elong) {
        float2* A = R2;
        float2* Bf = (R2 == X) ? Z : X;
        for (int q = tid; q < NFFT * NFFT; q += NT) A[q] = make_float2(A[q].x * A[q].x + A[q].y * A[q].y, 0.0f);
        __syncthreads();
        float2* S1 = stockham_fft(A, Bf, NFFT, rad, nr, NFFT, NFFT, 1, W, tid, NT);
        S1 = stockham_fft(S1, S1 == A ? Bf : A, NFFT, rad, nr, NFFT, 1, NFFT, W, tid, NT);
        for (int q = tid; q < NFFT * NFFT; q += NT) {
            const int kx = q % NFFT, ky = q / NFFT;
            const float ux = (float)(kx < NFFT / 2 ? kx : kx - NFFT), uy = (float)(ky < NFFT / 2 ? ky : ky - NFFT);
            const float d = ux * sd.dir_x + uy * sd.dir_y;
            const float o = expf(-sd.elong_a * d * d);
            S1[q] = make_float2(S1[q].x * o, -S1[q].y * o);
        }
        __syncthreads();
        float2* S2 = stockham_fft(S1, S1 == A ? Bf : A, NFFT, rad, nr, NFFT, NFFT, 1, W, tid, NT);
        img = stockham_fft(S2, S2 == A ? Bf : A, NFFT, rad, nr, NFFT, 1, NFFT, W, tid, NT);
    }

    // |.|^2 (or the elongated image), shift by NFFT/2, bin NBIN x NBIN
    const int lane = tid & 31, warp = tid >> 5;
    float b = 0.0f;
    const int o = tid;
    const int my = o / ND, mx = o % ND;
    if (o < ND * ND) {
        for (int ty = 0; ty < NBIN; ++ty)
            for (int tx = 0; tx < NBIN; ++tx) {
                int r = (my * NBIN + ty + NFFT / 2) % NFFT, c = (mx * NBIN + tx + NFFT / 2) % NFFT;
                const float2 v = img[r * NFFT + c];
                b += elong ? v.x : v.x * v.x + v.y * v.y;
            }
    }
    float s = warp_sum(b);
    if (lane == 0) red[warp] = s;
    __syncthreads();
    float bsum = 0.0f;
    for (int q = 0; q < NW; ++q) bsum += red[q];
    const float norm = (bsum > 0.0f) ? w.n_photons * sd.frac / bsum : 0.0f;
    __syncthreads();

    // pixel pairs (o, o + ND^2 / 2): the intensities go through shared memory (the spectrum
    // buffer, no longer read), the first ND^2 / 2 threads draw both pixels
    constexpr int HALF = ND * ND / 2;
    float* s_lam = reinterpret_cast<float*>(X);
    if (o < ND * ND) s_lam[o] = b * norm;
    __syncthreads();
    const float c0 = 0.5f * (float)(ND - 1);
    float sv = 0.0f, sx = 0.0f, sy = 0.0f;
    const long long pix0 = (long long)sd.rank * ND * ND;
    if (o < HALF) {
        const float lam_a = s_lam[o], lam_b = s_lam[o + HALF];
        float va = lam_a, vb = lam_b;
        if (L.ctx.noise) {
            int na, nb;
            noise_pair(lam_a, lam_b, w.read_noise, (uint32_t)(pix0 + o), (uint32_t)k, (uint32_t)w.wfs_index,
                       L.ctx.seed + real, recip, na, nb);
            va = (float)na;
            vb = (float)nb;
            if (L.frame_out) {
                L.frame_out[real * L.frame_stride + w.frame0 + pix0 + o] = na;
                L.frame_out[real * L.frame_stride + w.frame0 + pix0 + o + HALF] = nb;
            }
        }
        if (L.lam_out) {
            L.lam_out[real * L.frame_stride + w.frame0 + pix0 + o] = lam_a;
            L.lam_out[real * L.frame_stride + w.frame0 + pix0 + o + HALF] = lam_b;
        }
        const int my_b = (o + HALF) / ND;
        sv = va + vb;
        sx = ((float)mx - c0) * (va + vb);
        sy = fmaf((float)my_b - c0, vb, ((float)my - c0) * va);
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
        const float vx = gx - (L.s_ref ? L.s_ref[ix] : 0.0f), vy = gy - (L.s_ref ? L.s_ref[iy] : 0.0f);
        float* slopes = L.slopes + (long long)real * L.slope_stride;
        slopes[ix] = vx;
        slopes[iy] = vy;
        if (L.slopes_pad) {
            float* pad = L.slopes_pad + (long long)real * L.pad_stride;
            pad[w.rcol0 + sd.rank] = vx;
            pad[w.rcol0 + w.n_valid + sd.rank] = vy;
        }
    }
}

template <int NPX, int NFFT>
constexpr size_t fft_smem() {
    return sizeof(float2) * (2 * NFFT * NFFT + NFFT) + sizeof(AxisEnt) * 2 * kMaxEntries * NPX +
           sizeof(float) * (68 + 3 * (kFftThreads / 32));
}

// residual phase on the full pupil grid of one WFS, 8 x 8 tiles, one warp per tile
__global__ void __launch_bounds__(256) wfs_phase_kernel(Ctx ctx, int real, int wi, int N, float* out) {
    __shared__ AxisEnt s_ex[8][kMaxEntries * 8];
    __shared__ AxisEnt s_ey[8][kMaxEntries * 8];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int tiles_x = (N + 7) / 8;
    const int tile = blockIdx.x * 8 + warp;
    if (tile >= tiles_x * tiles_x) return;
    const int i0 = (tile % tiles_x) * 8, j0 = (tile / tiles_x) * 8;
    const GridView* V = ctx.views + real * ctx.view_stride + (long long)wi * ctx.n_grids;
    tile_entries<8>(V, ctx.n_grids, ctx.st->k, i0, j0, s_ex[warp], s_ey[warp], lane, 32);
    __syncwarp();
    for (int q = lane; q < 64; q += 32) {
        int x = q % 8, y = q / 8;
        if (i0 + x < N && j0 + y < N)
            out[(long long)(j0 + y) * N + i0 + x] = tile_phase(V, ctx.n_grids, s_ex[warp], s_ey[warp], 8, x, y);
    }
}

template <int NFFT, int NBIN>
cudaError_t launch_acf(const WfsLaunch& L, cudaStream_t s) {
    unsigned blocks = (unsigned)(((long long)L.n_subaps * L.ctx.n_real + 7) / 8);
    if (L.work && L.max_blocks > 0 && blocks > (unsigned)L.max_blocks) blocks = (unsigned)L.max_blocks;
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
    if (L.n_subaps) wfs_fft_kernel<NPX, NFFT, NBIN><<<(unsigned)(L.n_subaps * L.ctx.n_real), kFftThreads, sm, s>>>(L);
    return cudaGetLastError();
}

}  // namespace

bool wfs_variant_supported(int n_px, int n_fft, int n_bin, bool) {
    if (n_px == 8 && n_fft == 16 && n_bin == 2) return true;
    if (n_px == 8 && n_fft == 32 && n_bin == 2) return true;
    if (n_px == 8 && n_fft == 16 && n_bin == 1) return true;
    return wfs_variant_is_fft(n_px, n_fft, n_bin);
}

// block-per-subaperture variants: 2 x 2 low-order sensors (32 samples, FFT 64, bin 4) and
// laser stars with 16 samples per subaperture (twice the field of view of 8, FFT 32, bin 2)
bool wfs_variant_is_fft(int n_px, int n_fft, int n_bin) {
    return (n_px == 32 && n_fft == 64 && n_bin == 4) || (n_px == 16 && n_fft == 32 && n_bin == 2);
}

cudaError_t wfs_prepare() {
    cudaError_t e = prepare_fft<32, 64, 4>();
    return e == cudaSuccess ? prepare_fft<16, 32, 2>() : e;
}

cudaError_t launch_wfs(const WfsLaunch& L, int n_px, int n_fft, int n_bin, cudaStream_t s) {
    if (n_px == 8 && n_fft == 16 && n_bin == 2) return launch_acf<16, 2>(L, s);
    if (n_px == 8 && n_fft == 32 && n_bin == 2) return launch_acf<32, 2>(L, s);
    if (n_px == 8 && n_fft == 16 && n_bin == 1) return launch_acf<16, 1>(L, s);
    if (n_px == 32 && n_fft == 64 && n_bin == 4) return launch_fft<32, 64, 4>(L, s);
    if (n_px == 16 && n_fft == 32 && n_bin == 2) return launch_fft<16, 32, 2>(L, s);
    return cudaErrorInvalidValue;
}

cudaError_t launch_wfs_phase(const Ctx& ctx, int r, int wfs, int N, float* out, cudaStream_t s) {
    int tiles = ((N + 7) / 8) * ((N + 7) / 8);
    wfs_phase_kernel<<<(unsigned)((tiles + 7) / 8), 256, 0, s>>>(ctx, r, wfs, N, out);
    return cudaGetLastError();
}

}  // namespace mcao
