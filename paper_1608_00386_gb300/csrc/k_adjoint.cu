// Adjoint of the noise-free wavefront sensing: exact derivatives of the slopes with respect to
// the residual phase and to the DM commands ("The calibration of the interaction matrices":
// the interaction matrix is the slopes' response to each command; here it is the Jacobian at
// the current state rather than a finite poke).
//
// Forward model of one subaperture (the sensing step of "The closed loop"):
//   E(x) = A(x) exp(i (s phi(x) - pi (x + y) / N)) on the n_px^2 pupil samples, zero-padded to N,
//   F = FFT2(E), I = |F|^2, I' = M I with M = IFFT2 . diag(O_s) . FFT2 (sodium elongation; O_s the
//   OTF made even, (O(u) + O(-u)) / 2, which equals the forward's Re IFFT2(FFT2(I) O) for real
//   I), shift by N/2, bin b x b into det, CoG (sx, sy) = sum (m - c) det / sum det.
// Reverse pass for one slope (sx shown): g_det(m) = (m_x - c - sx) / T; unbin and unshift to g;
//   g <- M g (M is symmetric); H = sum_k g(k) F(k) exp(+2 pi i k.x / N) (unnormalized inverse DFT);
//   d sx / d phi(x) = -2 s Im(E(x) conj(H(x))).
// The x and y slopes of a subaperture share the forward pass; their adjoint images travel as the
// real and imaginary parts of one complex image through the (real) elongation operator.
//
// Projection on the DMs: phi(p) = ... - bilinear(S_m, p) and S_m = Gy C Gx^T, so
//   d phi(p) / d C[b][a] = -((1 - t_x) Gx[i0][a] + t_x Gx[i1][a]) ((1 - t_y) Gy[j0][b] + t_y Gy[j1][b]),
// the same fixed-point sample positions and clamped bilinear weights as the forward; actuators
// outside the union of the forward's per-tile bands (weights below 1e-10) are left out.  A
// rotated DM has no separable tables: its weights are evaluated at each bilinear corner.
#include "device_common.cuh"
#include "mcao_internal.h"

namespace mcao {

namespace {

constexpr int kAdjThreads = 256;
constexpr float kPi = 3.14159265358979323846f;
constexpr int kAdjMaxBand = 128;   // actuators per axis acting on one subaperture footprint

__device__ __forceinline__ float2* fft2_smem(float2* a, float2* b, int N, const int* rad, int nr, const float2* W,
                                             int tid, int nthr) {
    float2* r = stockham_fft(a, b, N, rad, nr, N, N, 1, W, tid, nthr);          // rows
    return stockham_fft(r, r == a ? b : a, N, rad, nr, N, 1, N, W, tid, nthr);  // columns
}

// even elongation OTF at frequency index (kx, ky): (O(u) + O(-u)) / 2, O(u) = exp(-a (u . d)^2),
// u the signed frequency of the index
__device__ __forceinline__ float otf_even(int kx, int ky, int N, float a, float dx, float dy) {
    const int ux = kx < N / 2 ? kx : kx - N, uy = ky < N / 2 ? ky : ky - N;
    const int mx = (N - kx) % N, my = (N - ky) % N;
    const int vx = mx < N / 2 ? mx : mx - N, vy = my < N / 2 ? my : my - N;
    const float d1 = (float)ux * dx + (float)uy * dy, d2 = (float)vx * dx + (float)vy * dy;
    return 0.5f * (expf(-a * d1 * d1) + expf(-a * d2 * d2));
}

// x <- M x = IFFT2(O_s FFT2(x)) for the image in a; returns the buffer holding the result
__device__ float2* elongate(float2* a, float2* b, int N, const int* rad, int nr, const float2* W, float ea, float dx,
                            float dy, int tid, int nthr) {
    float2* r = fft2_smem(a, b, N, rad, nr, W, tid, nthr);
    for (int q = tid; q < N * N; q += nthr) {
        const float o = otf_even(q % N, q / N, N, ea, dx, dy);
        r[q] = make_float2(r[q].x * o, -r[q].y * o);   // conj for the inverse by a forward FFT
    }
    __syncthreads();
    float2* r2 = fft2_smem(r, r == a ? b : a, N, rad, nr, W, tid, nthr);
    const float inv = 1.0f / (float)(N * N);
    for (int q = tid; q < N * N; q += nthr) r2[q] = make_float2(r2[q].x * inv, -r2[q].y * inv);
    __syncthreads();
    return r2;
}

__device__ __forceinline__ float block_sum(float v, float* red, int tid, int nthr) {
    v = warp_sum(v);
    if ((tid & 31) == 0) red[tid >> 5] = v;
    __syncthreads();
    float s = 0.0f;
    for (int q = 0; q < nthr / 32; ++q) s += red[q];
    __syncthreads();
    return s;
}

// One block per valid subaperture of one sensor: d s / d phi on its n_px^2 pupil samples for
// both of its slopes, rows slope0 + rank (x) and slope0 + n_valid + rank (y) of sens.
__global__ void __launch_bounds__(kAdjThreads) wfs_sens_kernel(SensLaunch L) {
    extern __shared__ float4 smem_raw[];
    const SubapDev sd = L.subaps[blockIdx.x];
    const WfsDev& w = L.ctx.wfs[sd.wfs];
    const int N = w.n_fft, npx = w.n_px, nb = w.n_bin, nd = w.n_det, NN = N * N;
    float2* E = reinterpret_cast<float2*>(smem_raw);
    float2* F = E + NN;
    float2* G = F + NN;
    float2* A = G + NN;
    float2* B = A + NN;
    float2* W = B + NN;
    float* red = reinterpret_cast<float*>(W + N);
    const int tid = threadIdx.x, nthr = blockDim.x;

    int rad[8];
    int nr = 0;
    for (int n = N; n > 1 && nr < 8;) {
        const int r = (n % 4 == 0) ? 4 : 2;
        rad[nr++] = r;
        n /= r;
    }
    for (int q = tid; q < N; q += nthr) {
        float s, c;
        sincospif(-2.0f * (float)q / (float)N, &s, &c);
        W[q] = make_float2(c, s);
    }
    for (int q = tid; q < NN; q += nthr) E[q] = make_float2(0.0f, 0.0f);
    __syncthreads();

    // forward: residual phase, field, spectrum
    const GridView* V = L.ctx.views + L.real * L.ctx.view_stride + (long long)sd.wfs * L.ctx.n_grids;
    const long long k = L.ctx.st->k;
    const int i0 = sd.sx * npx, j0 = sd.sy * npx;
    const float scale = w.scale;
    for (int q = tid; q < npx * npx; q += nthr) {
        const int x = q % npx, y = q / npx;
        float phi = 0.0f;
        for (int g = 0; g < L.ctx.n_grids; ++g) {
            const GridView& v = V[g];
            const AxisEnt ex = axis_entry(v.ax + (long long)(i0 + x) * v.bp + k * v.vx, v.n, v.periodic, v.inv_n);
            const AxisEnt ey = axis_entry(v.ay + (long long)(j0 + y) * v.bp + k * v.vy, v.n, v.periodic, v.inv_n);
            phi = fmaf(v.sign, bilinear(v.data, v.n, ex, ey), phi);
        }
        const float a = __ldg(w.amp + (long long)(j0 + y) * w.N + i0 + x);
        const float arg = scale * phi - kPi * (float)(x + y) / (float)N;
        float sn, cs;
        sincosf(arg, &sn, &cs);
        E[y * N + x] = make_float2(a * cs, a * sn);
    }
    __syncthreads();
    for (int q = tid; q < NN; q += nthr) A[q] = E[q];
    __syncthreads();
    {
        const float2* r = fft2_smem(A, B, N, rad, nr, W, tid, nthr);
        for (int q = tid; q < NN; q += nthr) F[q] = r[q];
    }
    __syncthreads();
    for (int q = tid; q < NN; q += nthr) A[q] = make_float2(F[q].x * F[q].x + F[q].y * F[q].y, 0.0f);
    __syncthreads();
    const bool elong = sd.elong_a > 0.0f;
    const float2* img = elong ? elongate(A, B, N, rad, nr, W, sd.elong_a, sd.dir_x, sd.dir_y, tid, nthr) : A;

    // binned detector image and its centre of gravity
    const float c0 = 0.5f * (float)(nd - 1);
    float tv = 0.0f, tx = 0.0f, ty = 0.0f;
    for (int m = tid; m < nd * nd; m += nthr) {
        const int my = m / nd, mx = m % nd;
        float b = 0.0f;
        for (int yy = 0; yy < nb; ++yy)
            for (int xx = 0; xx < nb; ++xx) {
                const int r = (my * nb + yy + N / 2) % N, c = (mx * nb + xx + N / 2) % N;
                b += img[r * N + c].x;
            }
        tv += b;
        tx += ((float)mx - c0) * b;
        ty += ((float)my - c0) * b;
    }
    tv = block_sum(tv, red, tid, nthr);
    tx = block_sum(tx, red, tid, nthr);
    ty = block_sum(ty, red, tid, nthr);
    const bool live = tv > 0.0f;
    const float inv_t = live ? 1.0f / tv : 0.0f;
    const float sx = tx * inv_t, sy = ty * inv_t;

    // adjoint image of the two slopes (x in the real part, y in the imaginary part), unbinned and
    // unshifted back to the spectrum's index order
    float2* g = (img == A) ? B : A;
    for (int q = tid; q < NN; q += nthr) {
        const int r = q / N, c = q % N;
        const int my = ((r + N / 2) % N) / nb, mx = ((c + N / 2) % N) / nb;
        g[q] = live ? make_float2(((float)mx - c0 - sx) * inv_t, ((float)my - c0 - sy) * inv_t) : make_float2(0.0f, 0.0f);
    }
    __syncthreads();
    if (elong) {
        const float2* r = elongate(g, g == A ? B : A, N, rad, nr, W, sd.elong_a, sd.dir_x, sd.dir_y, tid, nthr);
        for (int q = tid; q < NN; q += nthr) G[q] = r[q];
    } else {
        for (int q = tid; q < NN; q += nthr) G[q] = g[q];
    }
    __syncthreads();

    // per slope: H = unnormalized inverse DFT of g F = conj(FFT2(conj(g F))); d s / d phi
    const long long row_x = (long long)(w.slope0 + sd.rank) * L.P;
    const long long row_y = (long long)(w.slope0 + w.n_valid + sd.rank) * L.P;
    for (int part = 0; part < 2; ++part) {
        for (int q = tid; q < NN; q += nthr) {
            const float gv = part == 0 ? G[q].x : G[q].y;
            A[q] = make_float2(gv * F[q].x, -gv * F[q].y);
        }
        __syncthreads();
        const float2* h = fft2_smem(A, B, N, rad, nr, W, tid, nthr);   // conj(H)
        float* out = L.sens + (part == 0 ? row_x : row_y);
        for (int q = tid; q < npx * npx; q += nthr) {
            const int x = q % npx, y = q / npx;
            const float2 e = E[y * N + x], hc = h[y * N + x];
            // -2 s Im(E conj(H)), with hc = conj(H)
            out[q] = -2.0f * scale * (e.x * hc.y + e.y * hc.x);
        }
        __syncthreads();
    }
}

// Rotated DM: the weight of actuator (a, b) on surface sample (i, j) is the influence function
// at q(i, j) = R(-rot)((x_i, y_j) - shift) / mag; the slope's row entry sums the subaperture
// derivative over the four bilinear corners of every pupil sample.
__device__ void dm_adjoint_general(const ProjLaunch& L, const GridView& v, const DmDesc& dd, int row, int npx,
                                   const float* s_L, const AxisEnt* s_ex, const AxisEnt* s_ey, int* s_rng) {
    const int tid = threadIdx.x, nthr = blockDim.x;
    const float c0 = 0.5f * (float)(dd.surf_n - 1), ca = 0.5f * (float)(dd.nx - 1), cb = 0.5f * (float)(dd.ny - 1);
    auto to_act = [&](int i, int j, float& ua, float& ub) {
        const float x = ((float)i - c0) * dd.dx - dd.shx, y = ((float)j - c0) * dd.dx - dd.shy;
        ua = (dd.cr * x + dd.sr * y) * dd.inv_mag / dd.pitch + ca;
        ub = (-dd.sr * x + dd.cr * y) * dd.inv_mag / dd.pitch + cb;
    };
    if (tid == 0) {
        int cx0 = v.n, cx1 = 0, cy0 = v.n, cy1 = 0;
        for (int q = 0; q < npx; ++q) {
            cx0 = min(cx0, s_ex[q].idx & 0xffff);
            cx1 = max(cx1, s_ex[q].idx >> 16);
            cy0 = min(cy0, s_ey[q].idx & 0xffff);
            cy1 = max(cy1, s_ey[q].idx >> 16);
        }
        float lo_a = 1e30f, hi_a = -1e30f, lo_b = 1e30f, hi_b = -1e30f;
        for (int c = 0; c < 4; ++c) {
            float ua, ub;
            to_act((c & 1) ? cx1 : cx0, (c & 2) ? cy1 : cy0, ua, ub);
            lo_a = fminf(lo_a, ua); hi_a = fmaxf(hi_a, ua);
            lo_b = fminf(lo_b, ub); hi_b = fmaxf(hi_b, ub);
        }
        int a0 = max(0, (int)ceilf(lo_a - dd.rc)), a1 = min(dd.nx - 1, (int)floorf(hi_a + dd.rc)) + 1;
        int b0 = max(0, (int)ceilf(lo_b - dd.rc)), b1 = min(dd.ny - 1, (int)floorf(hi_b + dd.rc)) + 1;
        if (a1 < a0) a1 = a0;
        if (b1 < b0) b1 = b0;
        if (a1 - a0 > kAdjMaxBand || b1 - b0 > kAdjMaxBand) {
            atomicExch(L.err, 1);
            a1 = a0;
            b1 = b0;
        }
        s_rng[0] = a0; s_rng[1] = a1; s_rng[2] = b0; s_rng[3] = b1;
    }
    __syncthreads();
    const int a0 = s_rng[0], na = s_rng[1] - s_rng[0], b0 = s_rng[2], nbd = s_rng[3] - s_rng[2];
    for (int idx = tid; idx < na * nbd; idx += nthr) {
        const int b = idx / na, a = idx - b * na;
        const float fa = (float)(a0 + a), fb = (float)(b0 + b);
        float acc = 0.0f;
        for (int y = 0; y < npx; ++y) {
            const AxisEnt ey = s_ey[y];
            const int r0 = ey.idx & 0xffff, r1 = ey.idx >> 16;
            for (int x = 0; x < npx; ++x) {
                const float lv = s_L[y * npx + x];
                if (lv == 0.0f) continue;
                const AxisEnt ex = s_ex[x];
                const int q0 = ex.idx & 0xffff, q1 = ex.idx >> 16;
                float w = 0.0f;
                for (int c = 0; c < 4; ++c) {
                    const int i = (c & 1) ? q1 : q0, j = (c & 2) ? r1 : r0;
                    const float wc = ((c & 1) ? ex.t : 1.0f - ex.t) * ((c & 2) ? ey.t : 1.0f - ey.t);
                    float ua, ub;
                    to_act(i, j, ua, ub);
                    const float da = (ua - fa) * dd.pitch, db = (ub - fb) * dd.pitch;
                    w = fmaf(wc, expf(-(da * da + db * db) * dd.inv2s2), w);
                }
                acc = fmaf(lv, w, acc);
            }
        }
        const float val = v.sign * acc;
        const int cmd = L.act_map[dd.map_off + (long long)(b0 + b) * dd.nx + a0 + a];
        if (cmd < 0) continue;
        if (L.D) L.D[(long long)row * L.ld + cmd] = val;
        if (L.gc)
            for (int vv = 0; vv < L.n_vec; ++vv) {
                const float gv = L.gvec[(long long)vv * L.n_slopes + row];
                if (gv != 0.0f) atomicAdd(L.gc + (long long)vv * L.n_cmd + cmd, gv * val);
            }
    }
    __syncthreads();
}

// Gauss-Newton terms of a DM misregistration fit, one block per slope row of one sensor, for DM m
// only.  The row of the model matrix D(p) (the exact Jacobian with the DM moved by p = (shift_x,
// shift_y, rotation, magnification)) and its four derivatives dD/dp_i are formed by evaluating
// each actuator's influence function at the four bilinear corners of every pupil sample, in the
// DM's own frame (as the general adjoint does), and differentiating that evaluation:
//   u = R(-theta)(q - shift) / mag  (q a surface grid point, metres),  phi = exp(-|u - x_a|^2 / 2 s^2),
//   d phi / dp = -phi (u - x_a) . du/dp / s^2, with du/d shift_x = (-cos, sin) / mag,
//   du/d shift_y = (-sin, -cos) / mag, du/d theta = (B, -A) / mag, du/d mag = -(A, B) / mag^2
// (A, B the rotated offset before the division).  Against the measured row (columns of DM m) the
// block accumulates in double: cost = sum e^2 (e = D - D_meas), Jte_i = sum dD_i e, the upper
// triangle of JtJ_ij = sum dD_i dD_j, and sum D_meas^2; one record of 16 doubles per row.
__global__ void __launch_bounds__(256) misreg_gn_kernel(ProjLaunch L, int m, const float* __restrict__ D_meas,
                                                        long long ld_meas, int cmd0, double* __restrict__ rec) {
    __shared__ float s_L[kMaxNpx * kMaxNpx];
    __shared__ AxisEnt s_ex[kMaxNpx], s_ey[kMaxNpx];
    __shared__ int s_rng[4];
    __shared__ double s_red[8][16];
    const int tid = threadIdx.x, nthr = blockDim.x;
    const int axis = blockIdx.x / L.n_valid, rank = blockIdx.x - axis * L.n_valid;
    const SubapDev sd = L.subaps[rank];
    const WfsDev& w = L.ctx.wfs[sd.wfs];
    const int npx = w.n_px;
    const int row = w.slope0 + axis * w.n_valid + sd.rank;
    const int i0 = sd.sx * npx, j0 = sd.sy * npx;
    const GridView* V = L.ctx.views + L.real * L.ctx.view_stride + (long long)sd.wfs * L.ctx.n_grids;
    const long long k = L.ctx.st->k;
    for (int q = tid; q < npx * npx; q += nthr) s_L[q] = L.sens[(long long)row * L.P + q];
    const GridView& v = V[L.n_layers + m];
    const DmDesc dd = L.desc[m];
    if (tid < npx)
        s_ex[tid] = axis_entry(v.ax + (long long)(i0 + tid) * v.bp + k * v.vx, v.n, v.periodic, v.inv_n);
    else if (tid < 2 * npx)
        s_ey[tid - npx] = axis_entry(v.ay + (long long)(j0 + tid - npx) * v.bp + k * v.vy, v.n, v.periodic, v.inv_n);
    __syncthreads();
    const float c0 = 0.5f * (float)(dd.surf_n - 1), ca = 0.5f * (float)(dd.nx - 1), cb = 0.5f * (float)(dd.ny - 1);
    // offset of grid point (i, j) from the shift, rotated: (A, B), metres
    auto rot = [&](int i, int j, float& A, float& B) {
        const float x = ((float)i - c0) * dd.dx - dd.shx, y = ((float)j - c0) * dd.dx - dd.shy;
        A = dd.cr * x + dd.sr * y;
        B = -dd.sr * x + dd.cr * y;
    };
    if (tid == 0) {
        int cx0 = v.n, cx1 = 0, cy0 = v.n, cy1 = 0;
        for (int q = 0; q < npx; ++q) {
            cx0 = min(cx0, s_ex[q].idx & 0xffff);
            cx1 = max(cx1, s_ex[q].idx >> 16);
            cy0 = min(cy0, s_ey[q].idx & 0xffff);
            cy1 = max(cy1, s_ey[q].idx >> 16);
        }
        float lo_a = 1e30f, hi_a = -1e30f, lo_b = 1e30f, hi_b = -1e30f;
        for (int c = 0; c < 4; ++c) {
            float A, B;
            rot((c & 1) ? cx1 : cx0, (c & 2) ? cy1 : cy0, A, B);
            const float ua = A * dd.inv_mag / dd.pitch + ca, ub = B * dd.inv_mag / dd.pitch + cb;
            lo_a = fminf(lo_a, ua); hi_a = fmaxf(hi_a, ua);
            lo_b = fminf(lo_b, ub); hi_b = fmaxf(hi_b, ub);
        }
        int a0 = max(0, (int)ceilf(lo_a - dd.rc)), a1 = min(dd.nx - 1, (int)floorf(hi_a + dd.rc)) + 1;
        int b0 = max(0, (int)ceilf(lo_b - dd.rc)), b1 = min(dd.ny - 1, (int)floorf(hi_b + dd.rc)) + 1;
        if (a1 < a0) a1 = a0;
        if (b1 < b0) b1 = b0;
        s_rng[0] = a0; s_rng[1] = a1; s_rng[2] = b0; s_rng[3] = b1;
    }
    __syncthreads();
    const int a0 = s_rng[0], na = s_rng[1] - s_rng[0], b0 = s_rng[2], nbd = s_rng[3] - s_rng[2];
    const float im = dd.inv_mag, tws = 2.0f * dd.inv2s2;
    double acc[16];
#pragma unroll
    for (int q = 0; q < 16; ++q) acc[q] = 0.0;
    for (int idx = tid; idx < na * nbd; idx += nthr) {
        const int b = idx / na, a = idx - b * na;
        const int cmd = L.act_map[dd.map_off + (long long)(b0 + b) * dd.nx + a0 + a];
        if (cmd < 0) continue;
        const float xa = ((float)(a0 + a) - ca) * dd.pitch, yb = ((float)(b0 + b) - cb) * dd.pitch;
        float val = 0.0f, g0 = 0.0f, g1 = 0.0f, g2 = 0.0f, g3 = 0.0f;
        for (int y = 0; y < npx; ++y) {
            const AxisEnt ey = s_ey[y];
            const int r0 = ey.idx & 0xffff, r1 = ey.idx >> 16;
            for (int x = 0; x < npx; ++x) {
                const float lv = s_L[y * npx + x];
                if (lv == 0.0f) continue;
                const AxisEnt ex = s_ex[x];
                const int q0 = ex.idx & 0xffff, q1 = ex.idx >> 16;
                for (int c = 0; c < 4; ++c) {
                    const int i = (c & 1) ? q1 : q0, j = (c & 2) ? r1 : r0;
                    const float wl = lv * ((c & 1) ? ex.t : 1.0f - ex.t) * ((c & 2) ? ey.t : 1.0f - ey.t);
                    float A, B;
                    rot(i, j, A, B);
                    const float da = A * im - xa, db = B * im - yb;
                    const float ph = wl * expf(-(da * da + db * db) * dd.inv2s2);
                    val += ph;
                    const float gg = -tws * ph;   // d/dp of exp(-r^2 / 2 s^2) = -(r . dr/dp) / s^2 exp(..)
                    g0 = fmaf(gg, (-da * dd.cr + db * dd.sr) * im, g0);
                    g1 = fmaf(gg, (-da * dd.sr - db * dd.cr) * im, g1);
                    g2 = fmaf(gg, (da * B - db * A) * im, g2);
                    g3 = fmaf(gg, -(da * A + db * B) * im * im, g3);
                }
            }
        }
        const double dv = (double)(v.sign * val);
        const double d[4] = {(double)(v.sign * g0), (double)(v.sign * g1), (double)(v.sign * g2),
                             (double)(v.sign * g3)};
        const double meas = (double)D_meas[(long long)row * ld_meas + (cmd - cmd0)];
        const double e = dv - meas;
        acc[0] += e * e;
        acc[15] += meas * meas;
        int t = 5;
#pragma unroll
        for (int p = 0; p < 4; ++p) {
            acc[1 + p] += d[p] * e;
#pragma unroll
            for (int q = p; q < 4; ++q) acc[t++] += d[p] * d[q];
        }
    }
    // block sum in a fixed order: warp shuffles, then warp 0 over the warps
#pragma unroll
    for (int q = 0; q < 16; ++q)
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) acc[q] += __shfl_xor_sync(0xffffffffu, acc[q], o);
    const int lane = tid & 31, warp = tid >> 5;
    if (lane == 0)
#pragma unroll
        for (int q = 0; q < 16; ++q) s_red[warp][q] = acc[q];
    __syncthreads();
    if (tid < 16) {
        double sum = 0.0;
        for (int wv = 0; wv < (nthr >> 5); ++wv) sum += s_red[wv][tid];
        rec[(long long)row * 16 + tid] = sum;
    }
}

// rows' records summed in row order into out[16] (one block; fixed order)
__global__ void misreg_sum_kernel(const double* __restrict__ rec, int n_rows, double* __restrict__ out) {
    __shared__ double s[256];
    for (int q = 0; q < 16; ++q) {
        double sum = 0.0;
        for (int r = threadIdx.x; r < n_rows; r += blockDim.x) sum += rec[(long long)r * 16 + q];
        s[threadIdx.x] = sum;
        __syncthreads();
        if (threadIdx.x == 0) {
            double t = 0.0;
            for (int i = 0; i < (int)blockDim.x; ++i) t += s[i];
            out[q] = t;
        }
        __syncthreads();
    }
}

// One block per slope of one sensor: the slope's row of d s / d c from its pupil-sample
// derivatives, written to D (interaction matrix) and/or accumulated as g_v[row] * row into the
// command gradients of every vector v.
__global__ void __launch_bounds__(256) dm_adjoint_kernel(ProjLaunch L) {
    __shared__ float s_L[kMaxNpx * kMaxNpx];
    __shared__ float s_T[kAdjMaxBand * kMaxNpx];
    __shared__ float s_gy[kAdjMaxBand * kMaxNpx];
    __shared__ AxisEnt s_ex[kMaxNpx], s_ey[kMaxNpx];
    __shared__ int s_rng[4];
    const int tid = threadIdx.x, nthr = blockDim.x;
    const int axis = blockIdx.x / L.n_valid, rank = blockIdx.x - axis * L.n_valid;
    const SubapDev sd = L.subaps[rank];
    const WfsDev& w = L.ctx.wfs[sd.wfs];
    const int npx = w.n_px;
    const int row = w.slope0 + axis * w.n_valid + sd.rank;
    const int i0 = sd.sx * npx, j0 = sd.sy * npx;
    const GridView* V = L.ctx.views + L.real * L.ctx.view_stride + (long long)sd.wfs * L.ctx.n_grids;
    const long long k = L.ctx.st->k;
    for (int q = tid; q < npx * npx; q += nthr) s_L[q] = L.sens[(long long)row * L.P + q];
    for (int m = 0; m < L.n_dms; ++m) {
        const GridView& v = V[L.n_layers + m];
        const DmDesc dd = L.desc[m];
        if (tid < npx)
            s_ex[tid] = axis_entry(v.ax + (long long)(i0 + tid) * v.bp + k * v.vx, v.n, v.periodic, v.inv_n);
        else if (tid < 2 * npx)
            s_ey[tid - npx] = axis_entry(v.ay + (long long)(j0 + tid - npx) * v.bp + k * v.vy, v.n, v.periodic, v.inv_n);
        __syncthreads();
        if (dd.general) {
            dm_adjoint_general(L, v, dd, row, npx, s_L, s_ex, s_ey, s_rng);
            continue;
        }
        if (tid == 0) {
            int cx0 = v.n, cx1 = 0, cy0 = v.n, cy1 = 0;
            for (int q = 0; q < npx; ++q) {
                cx0 = min(cx0, s_ex[q].idx & 0xffff);
                cx1 = max(cx1, s_ex[q].idx >> 16);
                cy0 = min(cy0, s_ey[q].idx & 0xffff);
                cy1 = max(cy1, s_ey[q].idx >> 16);
            }
            // union of the forward's per-tile actuator bands over the tiles the footprint touches
            int a0 = dd.nx, a1 = 0, b0 = dd.ny, b1 = 0;
            for (int t = cx0 / kDmTile; t <= cx1 / kDmTile; ++t) {
                const int2 bt = L.band[dd.tband_x + t];
                if (bt.y > bt.x) { a0 = min(a0, bt.x); a1 = max(a1, bt.y); }
            }
            for (int t = cy0 / kDmTile; t <= cy1 / kDmTile; ++t) {
                const int2 bt = L.band[dd.tband_y + t];
                if (bt.y > bt.x) { b0 = min(b0, bt.x); b1 = max(b1, bt.y); }
            }
            if (a1 < a0) a1 = a0;
            if (b1 < b0) b1 = b0;
            if (a1 - a0 > kAdjMaxBand || b1 - b0 > kAdjMaxBand) {
                atomicExch(L.err, 1);
                a1 = a0;
                b1 = b0;
            }
            s_rng[0] = a0; s_rng[1] = a1; s_rng[2] = b0; s_rng[3] = b1;
        }
        __syncthreads();
        const int a0 = s_rng[0], na = s_rng[1] - s_rng[0], b0 = s_rng[2], nbd = s_rng[3] - s_rng[2];
        const float* Gx = L.g + dd.gx_off;
        const float* Gy = L.g + dd.gy_off;
        // T[a][y] = sum_x L[y][x] gx_a(x)
        for (int idx = tid; idx < na * npx; idx += nthr) {
            const int a = idx / npx, y = idx - a * npx;
            float acc = 0.0f;
            for (int x = 0; x < npx; ++x) {
                const AxisEnt e = s_ex[x];
                const int c0 = e.idx & 0xffff, c1 = e.idx >> 16;
                const float gxa = (1.0f - e.t) * Gx[(long long)c0 * dd.nx + a0 + a] + e.t * Gx[(long long)c1 * dd.nx + a0 + a];
                acc = fmaf(s_L[y * npx + x], gxa, acc);
            }
            s_T[a * npx + y] = acc;
        }
        for (int idx = tid; idx < nbd * npx; idx += nthr) {
            const int b = idx / npx, y = idx - b * npx;
            const AxisEnt e = s_ey[y];
            const int r0 = e.idx & 0xffff, r1 = e.idx >> 16;
            s_gy[b * npx + y] = (1.0f - e.t) * Gy[(long long)r0 * dd.ny + b0 + b] + e.t * Gy[(long long)r1 * dd.ny + b0 + b];
        }
        __syncthreads();
        for (int idx = tid; idx < na * nbd; idx += nthr) {
            const int b = idx / na, a = idx - b * na;
            float acc = 0.0f;
            for (int y = 0; y < npx; ++y) acc = fmaf(s_gy[b * npx + y], s_T[a * npx + y], acc);
            const float val = v.sign * acc;
            const int cmd = L.act_map[dd.map_off + (long long)(b0 + b) * dd.nx + a0 + a];
            if (cmd < 0) continue;
            if (L.D) L.D[(long long)row * L.ld + cmd] = val;
            if (L.gc)
                for (int vv = 0; vv < L.n_vec; ++vv) {
                    const float gv = L.gvec[(long long)vv * L.n_slopes + row];
                    if (gv != 0.0f) atomicAdd(L.gc + (long long)vv * L.n_cmd + cmd, gv * val);
                }
        }
        __syncthreads();
    }
}

// Per subaperture and vector: g_phi = g_v[x slope] L_x + g_v[y slope] L_y on its pupil samples,
// stored in g_phase[v][off + (j0 + y) N + i0 + x] and/or scattered onto the layers (the adjoint of
// the periodic bilinear sampling at the frozen-flow position of the step) in g_layers[v][...].
__global__ void phase_adjoint_kernel(ProjLaunch L, float* g_phase, long long phase_stride, long long phase_off,
                                     float* g_layers, long long layer_stride, const long long* layer_off) {
    const SubapDev sd = L.subaps[blockIdx.x];
    const WfsDev& w = L.ctx.wfs[sd.wfs];
    const int npx = w.n_px;
    const int rx = w.slope0 + sd.rank, ry = w.slope0 + w.n_valid + sd.rank;
    const int i0 = sd.sx * npx, j0 = sd.sy * npx;
    const GridView* V = L.ctx.views + L.real * L.ctx.view_stride + (long long)sd.wfs * L.ctx.n_grids;
    const long long k = L.ctx.st->k;
    for (int vv = 0; vv < L.n_vec; ++vv) {
        const float gx = L.gvec[(long long)vv * L.n_slopes + rx], gy = L.gvec[(long long)vv * L.n_slopes + ry];
        for (int q = threadIdx.x; q < npx * npx; q += blockDim.x) {
            const int x = q % npx, y = q / npx;
            const float gp = gx * L.sens[(long long)rx * L.P + q] + gy * L.sens[(long long)ry * L.P + q];
            if (g_phase) g_phase[vv * phase_stride + phase_off + (long long)(j0 + y) * w.N + i0 + x] = gp;
            if (!g_layers || gp == 0.0f) continue;
            for (int l = 0; l < L.n_layers; ++l) {
                const GridView& v = V[l];
                const AxisEnt ex = axis_entry(v.ax + (long long)(i0 + x) * v.bp + k * v.vx, v.n, v.periodic, v.inv_n);
                const AxisEnt ey = axis_entry(v.ay + (long long)(j0 + y) * v.bp + k * v.vy, v.n, v.periodic, v.inv_n);
                float* gl = g_layers + vv * layer_stride + layer_off[l];
                const int c0 = ex.idx & 0xffff, c1 = ex.idx >> 16, r0 = ey.idx & 0xffff, r1 = ey.idx >> 16;
                const float s = v.sign * gp;
                atomicAdd(gl + (long long)r0 * v.n + c0, s * (1.0f - ex.t) * (1.0f - ey.t));
                atomicAdd(gl + (long long)r0 * v.n + c1, s * ex.t * (1.0f - ey.t));
                atomicAdd(gl + (long long)r1 * v.n + c0, s * (1.0f - ex.t) * ey.t);
                atomicAdd(gl + (long long)r1 * v.n + c1, s * ex.t * ey.t);
            }
        }
    }
}

}  // namespace

size_t sens_smem(int n_fft) { return sizeof(float2) * (5 * (size_t)n_fft * n_fft + n_fft) + sizeof(float) * 32; }

cudaError_t launch_sens(const SensLaunch& L, int n_fft, cudaStream_t s) {
    const size_t bytes = sens_smem(n_fft);
    cudaError_t e = cudaFuncSetAttribute(wfs_sens_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
    if (e != cudaSuccess) return e;
    if (L.n_subaps) wfs_sens_kernel<<<(unsigned)L.n_subaps, kAdjThreads, bytes, s>>>(L);
    return cudaGetLastError();
}

cudaError_t launch_dm_adjoint(const ProjLaunch& L, cudaStream_t s) {
    if (L.n_valid && L.n_dms) dm_adjoint_kernel<<<(unsigned)(2 * L.n_valid), 256, 0, s>>>(L);
    return cudaGetLastError();
}

cudaError_t launch_misreg_gn(const ProjLaunch& L, int m, const float* D_meas, long long ld_meas, int cmd0, double* rec,
                             cudaStream_t s) {
    if (L.n_valid) misreg_gn_kernel<<<(unsigned)(2 * L.n_valid), 256, 0, s>>>(L, m, D_meas, ld_meas, cmd0, rec);
    return cudaGetLastError();
}

cudaError_t launch_misreg_sum(const double* rec, int n_rows, double* out, cudaStream_t s) {
    misreg_sum_kernel<<<1, 256, 0, s>>>(rec, n_rows, out);
    return cudaGetLastError();
}

cudaError_t launch_phase_adjoint(const ProjLaunch& L, float* g_phase, long long phase_stride, long long phase_off,
                                 float* g_layers, long long layer_stride, const long long* layer_off, cudaStream_t s) {
    if (L.n_valid)
        phase_adjoint_kernel<<<(unsigned)L.n_valid, 128, 0, s>>>(L, g_phase, phase_stride, phase_off, g_layers,
                                                                 layer_stride, layer_off);
    return cudaGetLastError();
}

}  // namespace mcao
