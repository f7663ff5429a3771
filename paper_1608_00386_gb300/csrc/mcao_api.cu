// Host side of libmcao: the C ABI declared in include/mcao.h.  Validates the configuration,
// derives geometry (pupils, valid subapertures, elongation, fixed-point projection maps,
// influence-function tables), owns the device state, and issues one closed-loop step as a CUDA
// graph whose branches overlap the ALU-bound sensing with the HBM-bound reconstructor product:
//   s0 (high priority): DM surfaces -> WFS kernel of sensor 0 -> sensor 1 -> ...
//   s1: block-per-subaperture WFS kernels (low-order sensors)
//   s3: reconstructor slice of sensor w as soon as sensor w's slopes exist, ..., reduction and
//       integrator
//   s2 (low priority): science field, row FFT (+ Strehl), column FFT (+ PSF accumulation)
// Every stage is a kernel of this library (k_dm.cu, k_wfs.cu, k_recon.cu, k_science.cu).
#include <cuda_runtime.h>

#include <algorithm>
#include <array>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <string>
#include <vector>

#include "../../include/mcao.h"
#include "mcao_internal.h"

using namespace mcao;

namespace {

thread_local std::string g_create_error;

struct Science {
    mcao_science p;
    int N, M;
    double dx, sum_amp;
    float* d_amp = nullptr;
    float2* d_field = nullptr;
    float2* d_ft = nullptr;
    double* d_psf_t = nullptr;
    float4* d_sr_part = nullptr;
    float2* d_w = nullptr;
    int n_tiles;
    std::vector<int> radices;
};

struct WfsHost {
    mcao_wfs p;
    int N, n_det, n_valid, slope0, frame0;
    int rcol0 = 0;                 // first column of this sensor's block in the padded R
    double dx;
    bool fft_route = false;
    std::vector<float> amp;
    std::vector<int> valid;        // subaperture index sy*n_sub+sx
    std::vector<double> frac;
    std::vector<SubapDev> subaps;
    SubapDev* d_subaps = nullptr;
};

struct FftGroup {                  // block-per-subaperture sensors sharing one kernel variant
    int n_px, n_fft, n_bin;
    std::vector<int> wfs;
    SubapDev* d_subaps = nullptr;
    int n_subaps = 0;
};

struct ProfSlot {                  // event-record nodes around one launch of one stage
    int stage;
    cudaEvent_t tpl_a = nullptr, tpl_b = nullptr;
    cudaGraphNode_t na = nullptr, nb = nullptr;
};

enum { ST_DM = MCAO_STAGE_DM, ST_WFS_MAIN = MCAO_STAGE_WFS_MAIN, ST_WFS_AUX = MCAO_STAGE_WFS_AUX,
       ST_RECON = MCAO_STAGE_RECON, ST_REDUCE = MCAO_STAGE_RECON_REDUCE, ST_SCIENCE = MCAO_STAGE_SCIENCE,
       ST_COUNT = MCAO_N_STAGES };

}  // namespace

struct mcao_sim {
    mcao_config cfg{};
    std::vector<WfsHost> wfs;
    std::vector<Science> sci;
    std::vector<FftGroup> fft_groups;
    std::string err;
    int device = 0, sm_count = 0;
    int n_slopes = 0, n_frame_px = 0, ld = 0;
    int n_real = 1;                       // realizations advanced together
    int cur = 0;                          // realization addressed by loads, getters and setters
    long long surf_total = 0;             // DM surface floats per realization

    cudaStream_t s0 = nullptr, s1 = nullptr, s2 = nullptr, s3 = nullptr;
    cudaStream_t user = nullptr;
    bool user_set = false;
    std::vector<cudaEvent_t> ev_pool;     // dependency events used while capturing
    cudaEvent_t ev_user = nullptr, ev_done = nullptr;
    // per-step readout (mcao_read_async): each read takes one slot of a device ring on s0 (a
    // small kernel after the queued steps), and the copies to the host run from that slot on
    // s_read, so that the next step does not wait behind them
    cudaStream_t s_read = nullptr;
    float* d_ring_c = nullptr;            // [kReadRing][ring_ncmd]
    double* d_ring_s = nullptr;           // [kReadRing][2 ring_nsci]
    int ring_ncmd = -1, ring_nsci = -1, ring_pos = 0;
    std::vector<cudaEvent_t> ring_ready, ring_free;   // per slot: snapshot written / copied out
    std::vector<char> ring_busy;

    // wfs
    WfsDev* d_wfs = nullptr;
    float* d_amp_all = nullptr;
    float* d_slopes = nullptr;
    float* d_slopes_pad = nullptr;        // slopes in R's padded column layout
    float* d_sref = nullptr;
    float* d_lam = nullptr;
    int* d_frames = nullptr;

    // atmosphere
    int n_layers = 0;
    std::vector<mcao_layer> layers;
    std::vector<float*> d_layer_owned;    // [n_real][n_layers], null where adopted
    std::vector<const float*> d_layer_ptr;   // [n_real][n_layers]
    std::vector<char> atm_loaded_r;       // per realization
    bool atm_loaded = false;              // every realization loaded

    // DMs
    int n_dms = 0;
    std::vector<mcao_dm> dms;
    std::vector<DmDesc> dm_desc;
    std::vector<int> dm_cmd0;          // first command of each DM (and the total)
    Tuning tune;                          // launch shapes (defaults or mcao_autotune's choice)
    std::vector<std::array<double, 4>> dm_misreg;   // per DM: shift x, y (m), rotation (rad), magnification
    DmDesc* d_dm_desc = nullptr;
    float* d_dm_g = nullptr;
    int dm_nb = 1;                        // largest actuator band of a 64 x 64 DM block (either axis)
    int2* d_dm_band = nullptr;
    int* d_dm_map = nullptr;
    float* d_dm_surf = nullptr;
    int dm_tile_start[kMaxDms + 1] = {0};
    int n_cmd = 0;
    bool dms_loaded = false;

    // grid views (layers then DMs) for every WFS and science direction
    GridView* d_views = nullptr;
    int n_grids = 0;

    // reconstructor
    unsigned char* d_R = nullptr;         // stage-tiled reconstructor (bytes, element format r_dtype)
    float* d_rscale = nullptr;            // per-row scales (FP8 E4M3)
    int r_dtype = 0;
    int rows_pad = 0;
    float* d_c = nullptr;
    float* d_partial = nullptr;
    // second-order controller (off: the pure integrator of gain cfg.gain)
    bool use_ctl = false;
    float ctl[4] = {1.0f, 0.0f, 0.0f, 0.0f};
    float* d_c_prev = nullptr;            // [n_real][n_cmd]
    float* d_dc_prev = nullptr;           // [n_real][n_cmd]
    float* d_dc = nullptr;                // [n_real][n_cmd] batched update (controller on)
    // batched product (n_real > 1).  float32 R: column-major [ld][rows_pad] copy streamed by the
    // CUDA-core product in groups of kMultiRhs realizations; bfloat16 R: the tensor-core product
    // (its own bfloat16 copy, split slopes and partials)
    float* d_Rrm = nullptr;
    float* d_multi_st = nullptr;          // float32 batched product: transposed slopes
    float* d_multi_part = nullptr;        // and split-K partials
    TcProduct* tc = nullptr;
    std::vector<ReconLaunch> slices;      // one per sensor with slopes
    std::vector<std::vector<int>> slice_wfs;  // sensors whose slopes each slice reads
    int n_chunks = 0;
    bool recon_loaded = false;

    StepState* d_st = nullptr;
    SciAcc* d_acc = nullptr;
    double* d_sr_out = nullptr;           // staging of mcao_read_async's Strehl ratios
    int* d_err = nullptr;                 // device-side error code (bounded waits)
    unsigned int* d_work = nullptr;       // work counters: [n_wfs] sensing launches, [n_wfs + 1] slices

    // graph
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t exec = nullptr;
    bool graph_dirty = true;
    unsigned int graph_mask = 0;          // stages whose event-record nodes the built graphs hold
    unsigned int capture_mask = 0;        // stages timed by the step being captured
    cudaGraph_t graph_k = nullptr;        // tune.steps_per_graph steps in one graph (profiler off)
    cudaGraphExec_t exec_k = nullptr;
    int graph_k_steps = 0;
    std::vector<ProfSlot> prof_slots;
    bool profiling = false;               // prof_mask != 0
    unsigned int prof_mask = 0;           // stages the profiler times (bit 1 << stage)
    std::vector<cudaEvent_t> prof_pool;
    size_t prof_used = 0;
    std::vector<std::pair<int, std::pair<cudaEvent_t, cudaEvent_t>>> prof_records;
    std::vector<size_t> prof_step_begin;  // index of each profiled step's first record
    int launches_per_step = 0;
};

namespace {

mcao_status fail(mcao_sim* s, mcao_status st, const char* fmt, ...) {
    char buf[512];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof(buf), fmt, ap);
    va_end(ap);
    if (s) s->err = buf;
    else g_create_error = buf;
    return st;
}

#define CK(expr)                                                                            \
    do {                                                                                    \
        cudaError_t e_ = (expr);                                                            \
        if (e_ != cudaSuccess) {                                                            \
            if (e_ == cudaErrorMemoryAllocation)                                            \
                return fail(S, MCAO_E_OOM, "%s: %s", #expr, cudaGetErrorString(e_));        \
            return fail(S, MCAO_E_CUDA, "%s: %s", #expr, cudaGetErrorString(e_));           \
        }                                                                                   \
    } while (0)

template <class T>
cudaError_t dalloc(T** p, size_t count) {
    if (count == 0) count = 1;
    return cudaMalloc((void**)p, sizeof(T) * count);
}

template <class T>
void dfree(T*& p) {
    if (p) cudaFree((void*)p);
    p = nullptr;
}

bool is_fin(double x) { return std::isfinite(x); }

long long to_q32(double v) { return std::llround(std::ldexp(v, 32)); }

// pupil amplitude on an n x n grid across D (sample i at (i - (n-1)/2) D/n), annulus rule
std::vector<float> pupil(double D, double obs, int n) {
    std::vector<float> A((size_t)n * n);
    double d = D / (double)n, R2 = 0.25 * D * D, ro2 = 0.25 * obs * obs * D * D;
    for (int j = 0; j < n; ++j)
        for (int i = 0; i < n; ++i) {
            double x = ((double)i - 0.5 * (double)(n - 1)) * d;
            double y = ((double)j - 0.5 * (double)(n - 1)) * d;
            double r2 = x * x + y * y;
            A[(size_t)j * n + i] = (r2 <= R2 && r2 >= ro2) ? 1.0f : 0.0f;
        }
    return A;
}

// elongation of one laser-star subaperture: FWHM b dh / H^2 rad along the launch-to-subaperture
// direction (b the distance from the launch), as the OTF factor exp(-elong_a (u . d)^2)
void set_elongation(const WfsHost& H, SubapDev& d) {
    d.elong_a = 0.0f;
    d.dir_x = d.dir_y = 0.0f;
    if (!(H.p.type == MCAO_WFS_LGS && H.p.na_fwhm > 0.0)) return;
    const int npx = H.p.n_px;
    const double pix_rad = H.p.lambda / ((double)H.p.n_fft * H.dx);
    const double cx = ((double)d.sx - 0.5 * (double)(H.p.n_sub - 1)) * npx * H.dx - H.p.launch_x;
    const double cy = ((double)d.sy - 0.5 * (double)(H.p.n_sub - 1)) * npx * H.dx - H.p.launch_y;
    const double b = std::sqrt(cx * cx + cy * cy);
    if (b > 0.0) {
        const double fwhm = b * H.p.na_fwhm / (H.p.height * H.p.height);
        const double sig = fwhm / (2.0 * std::sqrt(2.0 * std::log(2.0))) / pix_rad;
        d.elong_a = (float)(2.0 * M_PI * M_PI * sig * sig / ((double)H.p.n_fft * H.p.n_fft));
        d.dir_x = (float)(cx / b);
        d.dir_y = (float)(cy / b);
    }
}

std::vector<int> factor_fft(int M) {
    std::vector<int> r;
    int n = M;
    while (n % 4 == 0) { r.push_back(4); n /= 4; }
    while (n % 2 == 0) { r.push_back(2); n /= 2; }
    while (n % 5 == 0) { r.push_back(5); n /= 5; }
    while (n % 3 == 0) { r.push_back(3); n /= 3; }
    if (n != 1) r.clear();
    return r;
}

void release_graph(mcao_sim* S) {
    if (S->exec) cudaGraphExecDestroy(S->exec);
    if (S->graph) cudaGraphDestroy(S->graph);
    if (S->exec_k) cudaGraphExecDestroy(S->exec_k);
    if (S->graph_k) cudaGraphDestroy(S->graph_k);
    S->exec = nullptr;
    S->graph = nullptr;
    S->exec_k = nullptr;
    S->graph_k = nullptr;
    S->graph_k_steps = 0;
    S->graph_dirty = true;
    for (auto& p : S->prof_slots) {
        if (p.tpl_a) cudaEventDestroy(p.tpl_a);
        if (p.tpl_b) cudaEventDestroy(p.tpl_b);
    }
    S->prof_slots.clear();
}

int pad_stride(const mcao_sim* S) { return S->ld + kSlopePadTail; }

Ctx make_ctx(mcao_sim* S) {
    Ctx c;
    c.views = S->d_views;
    c.n_grids = S->n_grids;
    c.view_stride = (long long)(S->wfs.size() + S->sci.size()) * S->n_grids;
    c.n_real = S->n_real;
    c.wfs = S->d_wfs;
    c.st = S->d_st;
    c.seed = S->cfg.seed;
    c.noise = S->cfg.noise;
    return c;
}

DmLaunch make_dm_launch(mcao_sim* S) {
    DmLaunch L{};
    L.n_dm = S->n_dms;
    for (int m = 0; m < S->n_dms && m < kMaxDms; ++m) L.desc[m] = S->dm_desc[m];
    L.nb = S->dm_nb;
    L.g = S->d_dm_g;
    L.band = S->d_dm_band;
    L.act_map = S->d_dm_map;
    L.c = S->d_c;
    L.surf = S->d_dm_surf;
    L.n_real = S->n_real;
    L.n_cmd = S->n_cmd;
    L.surf_stride = S->surf_total;
    for (int m = 0; m <= kMaxDms; ++m) L.tile_start[m] = S->dm_tile_start[m];
    L.st = S->d_st;
    L.work = S->d_work;
    L.n_work = (int)(S->wfs.size() + S->slices.size());
    return L;
}

SciLaunch make_sci_launch(mcao_sim* S, int q) {
    Science& C = S->sci[q];
    SciLaunch L{};
    L.ctx = make_ctx(S);
    L.view = (int)S->wfs.size() + q;
    L.N = C.N;
    L.M = C.M;
    L.scale = (float)(S->cfg.lambda_ref / C.p.lambda);
    L.amp = C.d_amp;
    L.field = C.d_field;
    L.ft = C.d_ft;
    L.psf_t = C.d_psf_t;
    L.sr_part = C.d_sr_part;
    L.n_tiles = C.n_tiles;
    L.sum_amp = C.sum_amp;
    L.psf_every = S->cfg.psf_every;
    L.w = C.d_w;
    L.n_radices = (int)C.radices.size();
    for (int i = 0; i < L.n_radices && i < 8; ++i) L.radices[i] = C.radices[i];
    L.st = S->d_st;
    L.acc = S->d_acc + q;
    L.acc_stride = (int)S->sci.size();
    return L;
}

WfsLaunch make_wfs_launch(mcao_sim* S, const SubapDev* subaps, int n, unsigned int* work = nullptr) {
    WfsLaunch L{};
    L.work = work;
    L.max_blocks = S->tune.sense_blocks_per_sm * S->sm_count;  // warp-per-subaperture blocks per SM
    L.ctx = make_ctx(S);
    L.subaps = subaps;
    L.n_subaps = n;
    L.s_ref = S->d_sref;
    L.slopes = S->d_slopes;
    L.slopes_pad = S->d_slopes_pad;
    L.lam_out = S->cfg.keep_frames ? S->d_lam : nullptr;
    L.frame_out = (S->cfg.keep_frames && S->cfg.noise) ? S->d_frames : nullptr;
    L.slope_stride = S->n_slopes;
    L.pad_stride = pad_stride(S);
    L.frame_stride = S->n_frame_px;
    return L;
}

// Fixed-point projection maps of every grid (layers, then DMs) for every view (WFSs, then
// science directions): a pupil sample x of a view with N samples across D at height H maps to
// the grid index (x (1 - h/H) + h theta + (k dt) v) / pixel + (n - 1)/2.
mcao_status rebuild_views(mcao_sim* S) {
    struct G { int n, periodic; double pixel, alt, vx, vy; float sign; };
    std::vector<G> grids;
    for (int l = 0; l < S->n_layers; ++l) {
        const mcao_layer& L = S->layers[l];
        grids.push_back({L.n, 1, L.pixel_m, L.alt_m, L.vx, L.vy, 1.0f});
    }
    for (int m = 0; m < S->n_dms; ++m) {
        const mcao_dm& d = S->dms[m];
        grids.push_back({d.surf_n, 0, d.surf_dx, d.alt_m, 0.0, 0.0, -1.0f});
    }
    // data of grid g for realization r
    auto grid_data = [&](int r, int g) -> const float* {
        if (g < S->n_layers) {
            const size_t i = (size_t)r * S->n_layers + g;
            return i < S->d_layer_ptr.size() ? S->d_layer_ptr[i] : nullptr;
        }
        const int m = g - S->n_layers;
        return S->d_dm_surf ? S->d_dm_surf + (size_t)r * S->surf_total + S->dm_desc[m].surf_off : nullptr;
    };
    if ((int)grids.size() > kMaxEntries)
        return fail(S, MCAO_E_UNSUPPORTED, "layers + DMs = %d exceeds %d", (int)grids.size(), kMaxEntries);
    struct View { int N; double thx, thy, H; };
    std::vector<View> views;
    for (const auto& w : S->wfs)
        views.push_back({w.N, w.p.theta_x, w.p.theta_y, w.p.type == MCAO_WFS_LGS ? w.p.height : 0.0});
    for (const auto& c : S->sci) views.push_back({c.N, c.p.theta_x, c.p.theta_y, 0.0});
    std::vector<GridView> out;
    const double D = S->cfg.D, dt = S->cfg.dt;
    for (int r = 0; r < S->n_real; ++r)
    for (const auto& v : views) {
        const double dxp = D / (double)v.N;
        for (size_t gi = 0; gi < grids.size(); ++gi) {
            const G& g = grids[gi];
            double f = (v.H > 0.0) ? 1.0 - g.alt / v.H : 1.0;
            double x0 = (0.0 - 0.5 * (double)(v.N - 1)) * dxp * f;
            GridView gv{};
            gv.data = grid_data(r, (int)gi);
            gv.n = g.n;
            gv.periodic = g.periodic;
            gv.ax = to_q32((x0 + g.alt * v.thx) / g.pixel + 0.5 * (double)(g.n - 1));
            gv.ay = to_q32((x0 + g.alt * v.thy) / g.pixel + 0.5 * (double)(g.n - 1));
            gv.bp = to_q32(dxp * f / g.pixel);
            gv.vx = to_q32(dt * g.vx / g.pixel);
            gv.vy = to_q32(dt * g.vy / g.pixel);
            gv.sign = g.sign;
            gv.inv_n = (float)(1.0 / (double)g.n);
            out.push_back(gv);
        }
    }
    dfree(S->d_views);
    S->n_grids = (int)grids.size();
    CK(dalloc(&S->d_views, out.size()));
    if (!out.empty()) CK(cudaMemcpyAsync(S->d_views, out.data(), sizeof(GridView) * out.size(), cudaMemcpyHostToDevice, S->s0));
    release_graph(S);
    CK(cudaStreamSynchronize(S->s0));
    return MCAO_OK;
}

// ---------------------------------------------------------------------------------------------
// step issue
// ---------------------------------------------------------------------------------------------
cudaEvent_t dep_event(mcao_sim* S, size_t& used) {
    if (used >= S->ev_pool.size()) {
        cudaEvent_t e = nullptr;
        cudaEventCreateWithFlags(&e, cudaEventDisableTiming);
        S->ev_pool.push_back(e);
    }
    return S->ev_pool[used++];
}

// profiling: an event-record node before and after a launch, present only in graphs captured
// with the profiler on (each node is a dependency hop between the kernels it separates)
int prof_begin(mcao_sim* S, int stage, cudaStream_t st) {
    if (!(S->capture_mask & (1u << stage))) return -1;
    ProfSlot p;
    p.stage = stage;
    cudaEventCreate(&p.tpl_a);
    cudaEventCreate(&p.tpl_b);
    cudaEventRecordWithFlags(p.tpl_a, st, cudaEventRecordExternal);
    S->prof_slots.push_back(p);
    return (int)S->prof_slots.size() - 1;
}

void prof_end(mcao_sim* S, int slot, cudaStream_t st) {
    if (slot < 0) return;
    cudaEventRecordWithFlags(S->prof_slots[slot].tpl_b, st, cudaEventRecordExternal);
}

// Queue one step (captured into the graph).  Returns the first launch error.
// Product of the first n realizations' padded slopes with the shared R:
// out[r][i] = alpha sum_j R[i][j] s_r[j] + beta out[r][i], on s0.  bfloat16 R runs on the tensor
// cores (64 realizations per pass over R), float32 R on the CUDA-core kernel (kMultiRhs per pass).
cudaError_t enqueue_batched_product(mcao_sim* S, int n, float alpha, float beta, float* out, int* nl) {
    cudaError_t e = cudaSuccess;
    if (S->tc) {
        int n_tc = 0;
        if ((e = tc_launch(S->tc, S->d_slopes_pad, pad_stride(S), n, alpha, beta, out, S->d_err, S->tune.tc_chunk,
                           S->s0, &n_tc)) != cudaSuccess)
            return e;
        *nl += n_tc;
        return cudaSuccess;
    }
    MultiLaunch M{};
    M.R = S->d_Rrm;
    M.bf16 = 0;
    M.rows_pad = S->rows_pad;
    M.n_cmd = S->n_cmd;
    M.K = S->ld;
    M.s_t = S->d_multi_st;
    M.partial = S->d_multi_part;
    for (int r0 = 0; r0 < n; r0 += kMultiRhs) {
        const int nb = std::min(kMultiRhs, n - r0);
        if ((e = launch_recon_multi(M, nb, pad_stride(S), S->d_slopes_pad + (size_t)r0 * pad_stride(S), alpha, beta,
                                    out + (size_t)r0 * S->n_cmd, S->sm_count, S->tune.multi_blocks_per_sm, S->s0)) !=
            cudaSuccess)
            return e;
        *nl += 3;
    }
    return cudaSuccess;
}

cudaError_t enqueue_step(mcao_sim* S, int* launches) {
    cudaError_t e;
    int nl = 0;
    size_t used = 0;
    int slot = prof_begin(S, ST_DM, S->s0);
    if ((e = launch_dm_surfaces(make_dm_launch(S), S->s0)) != cudaSuccess) return e;
    nl += 1;
    prof_end(S, slot, S->s0);
    cudaEvent_t ev_fork = dep_event(S, used);
    if ((e = cudaEventRecord(ev_fork, S->s0)) != cudaSuccess) return e;
    for (cudaStream_t st : {S->s1, S->s2, S->s3})
        if ((e = cudaStreamWaitEvent(st, ev_fork, 0)) != cudaSuccess) return e;

    // block-per-subaperture sensors on s1
    std::vector<cudaEvent_t> ready(S->wfs.size(), nullptr);
    for (const auto& g : S->fft_groups) {
        slot = prof_begin(S, ST_WFS_AUX, S->s1);
        if ((e = launch_wfs(make_wfs_launch(S, g.d_subaps, g.n_subaps), g.n_px, g.n_fft, g.n_bin, S->s1)) != cudaSuccess)
            return e;
        prof_end(S, slot, S->s1);
        ++nl;
        cudaEvent_t ev = dep_event(S, used);
        if ((e = cudaEventRecord(ev, S->s1)) != cudaSuccess) return e;
        for (int w : g.wfs) ready[w] = ev;
    }

    // science on s2 (low priority): after the block-per-subaperture sensors, so that it fills
    // the SMs the first warp-per-subaperture launch leaves rather than racing it for them
    {
        cudaEvent_t after = nullptr;
        for (cudaEvent_t ev : ready)
            if (ev) after = ev;
        if (S->tune.science_after_aux && after && (e = cudaStreamWaitEvent(S->s2, after, 0)) != cudaSuccess)
            return e;
    }
    for (size_t q = 0; q < S->sci.size(); ++q) {
        SciLaunch L = make_sci_launch(S, (int)q);
        slot = prof_begin(S, ST_SCIENCE, S->s2);
        if ((e = launch_sci_field(L, S->s2)) != cudaSuccess) return e;
        if ((e = launch_sci_rows(L, S->s2)) != cudaSuccess) return e;
        if ((e = launch_sci_cols(L, S->s2)) != cudaSuccess) return e;
        prof_end(S, slot, S->s2);
        nl += 3;
    }
    cudaEvent_t ev_sci = dep_event(S, used);
    if ((e = cudaEventRecord(ev_sci, S->s2)) != cudaSuccess) return e;

    // warp-per-subaperture sensors, one launch each, on s0
    for (size_t w = 0; w < S->wfs.size(); ++w) {
        const WfsHost& W = S->wfs[w];
        if (W.fft_route || W.n_valid == 0) continue;
        slot = prof_begin(S, ST_WFS_MAIN, S->s0);
        if ((e = launch_wfs(make_wfs_launch(S, W.d_subaps, W.n_valid, S->d_work + w), W.p.n_px, W.p.n_fft,
                            W.p.n_bin, S->s0)) != cudaSuccess)
            return e;
        prof_end(S, slot, S->s0);
        ++nl;
        cudaEvent_t ev = dep_event(S, used);
        if ((e = cudaEventRecord(ev, S->s0)) != cudaSuccess) return e;
        ready[w] = ev;
    }

    if (S->n_real > 1) {
        // batched: after every sensor of every realization, C += g R S for all realizations at
        // once (one pass over R), then the step counter
        cudaEvent_t ev_s1b = dep_event(S, used);
        if ((e = cudaEventRecord(ev_s1b, S->s1)) != cudaSuccess) return e;
        if ((e = cudaStreamWaitEvent(S->s0, ev_s1b, 0)) != cudaSuccess) return e;
        slot = prof_begin(S, ST_RECON, S->s0);
        // integrator: C += g R S in place; controller: D = R S, then the filter
        const float alpha = S->use_ctl ? 1.0f : (float)S->cfg.gain, beta = S->use_ctl ? 0.0f : 1.0f;
        if ((e = enqueue_batched_product(S, S->n_real, alpha, beta, S->use_ctl ? S->d_dc : S->d_c, &nl)) != cudaSuccess)
            return e;
        prof_end(S, slot, S->s0);
        ReduceLaunch fin{S->use_ctl ? S->n_cmd : 0, 0, nullptr, S->d_c, 0.0f, S->d_st};
        fin.use_ctl = S->use_ctl;
        fin.a1 = S->ctl[0]; fin.a2 = S->ctl[1]; fin.b0 = S->ctl[2]; fin.b1 = S->ctl[3];
        fin.c_prev = S->d_c_prev;
        fin.dc_prev = S->d_dc_prev;
        fin.dc_in = S->d_dc;
        fin.n_real = S->n_real;
        if ((e = launch_recon_reduce(fin, S->s0)) != cudaSuccess) return e;
        nl += 2;
        if ((e = cudaStreamWaitEvent(S->s0, ev_sci, 0)) != cudaSuccess) return e;
        cudaEvent_t ev_s3 = dep_event(S, used);   // s3 forked: join it back untouched
        if ((e = cudaEventRecord(ev_s3, S->s3)) != cudaSuccess) return e;
        if ((e = cudaStreamWaitEvent(S->s0, ev_s3, 0)) != cudaSuccess) return e;
        if (launches) *launches = nl;
        return cudaSuccess;
    }

    // reconstructor slices on s3, each after its sensor, then the reduction
    ReduceLaunch rl{S->n_cmd, S->n_chunks, S->d_partial, S->d_c, (float)S->cfg.gain, S->d_st};
    rl.use_ctl = S->use_ctl;
    rl.a1 = S->ctl[0]; rl.a2 = S->ctl[1]; rl.b0 = S->ctl[2]; rl.b1 = S->ctl[3];
    rl.c_prev = S->d_c_prev;
    rl.dc_prev = S->d_dc_prev;
    rl.n_real = 1;
    for (size_t i = 0; i < S->slices.size(); ++i) {
        cudaEvent_t last = nullptr;
        for (int w : S->slice_wfs[i]) {
            cudaEvent_t ev = ready[w];
            if (ev && ev != last && (e = cudaStreamWaitEvent(S->s3, ev, 0)) != cudaSuccess) return e;
            last = ev;
        }
        slot = prof_begin(S, ST_RECON, S->s3);
        ReconLaunch rl_i = S->slices[i];
        rl_i.max_ctas = std::max(1, S->sm_count * S->tune.recon_ctas_pct / 100);
        // the last slice follows the last sensor and has the SMs to itself: one block per SM
        if (i + 1 == S->slices.size()) rl_i.max_ctas = std::max(rl_i.max_ctas, S->sm_count);
        if ((e = launch_recon(rl_i, S->s3)) != cudaSuccess) return e;
        prof_end(S, slot, S->s3);
        ++nl;
    }
    slot = prof_begin(S, ST_REDUCE, S->s3);
    if ((e = launch_recon_reduce(rl, S->s3)) != cudaSuccess) return e;
    prof_end(S, slot, S->s3);
    ++nl;

    // join every branch back into s0
    cudaEvent_t ev_gemv = dep_event(S, used);
    if ((e = cudaEventRecord(ev_gemv, S->s3)) != cudaSuccess) return e;
    cudaEvent_t ev_s1 = dep_event(S, used);
    if ((e = cudaEventRecord(ev_s1, S->s1)) != cudaSuccess) return e;
    for (cudaEvent_t ev : {ev_gemv, ev_sci, ev_s1})
        if ((e = cudaStreamWaitEvent(S->s0, ev, 0)) != cudaSuccess) return e;
    if (launches) *launches = nl;
    return cudaSuccess;
}

// capture n consecutive steps into one graph (the streams join back into s0 after each step)
static mcao_status capture_steps(mcao_sim* S, int n, cudaGraph_t* out, int* launches) {
    CK(cudaStreamBeginCapture(S->s0, cudaStreamCaptureModeThreadLocal));
    cudaError_t e = cudaSuccess;
    for (int i = 0; i < n && e == cudaSuccess; ++i) e = enqueue_step(S, launches);
    cudaGraph_t g = nullptr;
    cudaError_t e2 = cudaStreamEndCapture(S->s0, &g);
    if (e != cudaSuccess) {
        if (g) cudaGraphDestroy(g);
        return fail(S, MCAO_E_CUDA, "step capture: %s", cudaGetErrorString(e));
    }
    if (e2 != cudaSuccess) return fail(S, MCAO_E_CUDA, "end capture: %s", cudaGetErrorString(e2));
    *out = g;
    return MCAO_OK;
}

mcao_status build_graph(mcao_sim* S) {
    release_graph(S);
    int nl = 0;
    S->capture_mask = S->prof_mask;
    mcao_status r = capture_steps(S, 1, &S->graph, &nl);
    S->capture_mask = 0;
    if (r != MCAO_OK) return r;
    S->graph_mask = S->prof_mask;
    CK(cudaGraphInstantiate(&S->exec, S->graph, cudaGraphInstantiateFlagUseNodePriority));
    // locate the profiling event-record nodes
    size_t n = 0;
    CK(cudaGraphGetNodes(S->graph, nullptr, &n));
    std::vector<cudaGraphNode_t> nodes(n);
    CK(cudaGraphGetNodes(S->graph, nodes.data(), &n));
    for (size_t i = 0; i < n; ++i) {
        cudaGraphNodeType t;
        CK(cudaGraphNodeGetType(nodes[i], &t));
        if (t != cudaGraphNodeTypeEventRecord) continue;
        cudaEvent_t ev;
        CK(cudaGraphEventRecordNodeGetEvent(nodes[i], &ev));
        for (auto& p : S->prof_slots) {
            if (p.tpl_a == ev) p.na = nodes[i];
            if (p.tpl_b == ev) p.nb = nodes[i];
        }
    }
    S->launches_per_step = nl;
    // several steps per graph launch when the profiler is off: the steps inside one graph follow
    // one another through plain graph edges instead of a graph launch boundary each
    if (!S->profiling && S->tune.steps_per_graph > 1) {
        int nk = 0;
        r = capture_steps(S, S->tune.steps_per_graph, &S->graph_k, &nk);
        if (r != MCAO_OK) return r;
        CK(cudaGraphInstantiate(&S->exec_k, S->graph_k, cudaGraphInstantiateFlagUseNodePriority));
        S->graph_k_steps = S->tune.steps_per_graph;
    }
    S->graph_dirty = false;
    return MCAO_OK;
}

mcao_status order_after_user(mcao_sim* S) {
    if (!S->user_set) return MCAO_OK;
    CK(cudaEventRecord(S->ev_user, S->user));
    CK(cudaStreamWaitEvent(S->s0, S->ev_user, 0));
    return MCAO_OK;
}

mcao_status signal_user(mcao_sim* S) {
    if (!S->user_set) return MCAO_OK;
    CK(cudaEventRecord(S->ev_done, S->s0));
    CK(cudaStreamWaitEvent(S->user, S->ev_done, 0));
    return MCAO_OK;
}

mcao_status sync_all(mcao_sim* S) {
    for (cudaStream_t st : {S->s0, S->s1, S->s2, S->s3}) CK(cudaStreamSynchronize(st));
    if (S->s_read) CK(cudaStreamSynchronize(S->s_read));
    if (S->d_err) {
        int e = 0;
        CK(cudaMemcpy(&e, S->d_err, sizeof(int), cudaMemcpyDeviceToHost));
        if (e != 0) {
            CK(cudaMemsetAsync(S->d_err, 0, sizeof(int), S->s0));
            return fail(S, MCAO_E_TIMEOUT, "a bounded device wait gave up (code %d): results of the last steps are invalid",
                        e);
        }
    }
    return MCAO_OK;
}

void destroy_all(mcao_sim* S) {
    if (!S) return;
    cudaSetDevice(S->device);
    for (cudaStream_t st : {S->s0, S->s1, S->s2, S->s3})
        if (st) cudaStreamSynchronize(st);
    release_graph(S);
    for (auto& w : S->wfs) dfree(w.d_subaps);
    for (auto& g : S->fft_groups) dfree(g.d_subaps);
    for (auto& c : S->sci) {
        dfree(c.d_amp); dfree(c.d_field); dfree(c.d_ft); dfree(c.d_psf_t); dfree(c.d_sr_part); dfree(c.d_w);
    }
    dfree(S->d_wfs); dfree(S->d_amp_all); dfree(S->d_slopes); dfree(S->d_slopes_pad); dfree(S->d_sref);
    dfree(S->d_lam);
    dfree(S->d_frames);
    for (auto p : S->d_layer_owned)
        if (p) cudaFree(p);
    S->d_layer_owned.clear();
    dfree(S->d_dm_desc); dfree(S->d_dm_g); dfree(S->d_dm_band); dfree(S->d_dm_map);
    dfree(S->d_dm_surf); dfree(S->d_views); dfree(S->d_R); dfree(S->d_rscale); dfree(S->d_c); dfree(S->d_partial);
    dfree(S->d_st); dfree(S->d_acc); dfree(S->d_err); dfree(S->d_work); dfree(S->d_sr_out);
    dfree(S->d_Rrm);
    dfree(S->d_c_prev); dfree(S->d_dc_prev); dfree(S->d_dc);
    tc_destroy(S->tc);
    dfree(S->d_multi_st); dfree(S->d_multi_part);
    for (auto e : S->prof_pool) cudaEventDestroy(e);
    for (auto e : S->ev_pool) cudaEventDestroy(e);
    for (cudaEvent_t e : {S->ev_user, S->ev_done})
        if (e) cudaEventDestroy(e);
    dfree(S->d_ring_c); dfree(S->d_ring_s);
    for (auto e : S->ring_ready) cudaEventDestroy(e);
    for (auto e : S->ring_free) cudaEventDestroy(e);
    for (cudaStream_t st : {S->s0, S->s1, S->s2, S->s3, S->s_read})
        if (st) cudaStreamDestroy(st);
    delete S;
}

mcao_status validate_config(const mcao_config* c) {
    mcao_sim* S = nullptr;
    if (!c) return fail(S, MCAO_E_INVALID_ARG, "cfg is NULL");
    if (c->struct_size != sizeof(mcao_config))
        return fail(S, MCAO_E_INVALID_ARG, "struct_size %zu != %zu", c->struct_size, sizeof(mcao_config));
    if (!(is_fin(c->D) && c->D > 0)) return fail(S, MCAO_E_INVALID_ARG, "D must be > 0");
    if (!(is_fin(c->obstruction) && c->obstruction >= 0 && c->obstruction < 1))
        return fail(S, MCAO_E_INVALID_ARG, "obstruction must be in [0, 1)");
    if (!(is_fin(c->lambda_ref) && c->lambda_ref > 0)) return fail(S, MCAO_E_INVALID_ARG, "lambda_ref must be > 0");
    if (!(is_fin(c->dt) && c->dt >= 0)) return fail(S, MCAO_E_INVALID_ARG, "dt must be >= 0");
    if (!is_fin(c->gain)) return fail(S, MCAO_E_INVALID_ARG, "gain must be finite");
    if (c->psf_every < 0) return fail(S, MCAO_E_INVALID_ARG, "psf_every must be >= 0");
    if (c->n_real < 1 || c->n_real > 4096) return fail(S, MCAO_E_INVALID_ARG, "n_real must be in [1, 4096]");
    if (c->n_wfs < 1 || !c->wfs) return fail(S, MCAO_E_INVALID_ARG, "at least one WFS is required");
    if (c->n_sci < 0 || (c->n_sci > 0 && !c->sci)) return fail(S, MCAO_E_INVALID_ARG, "bad science list");
    for (int w = 0; w < c->n_wfs; ++w) {
        const mcao_wfs& p = c->wfs[w];
        if (p.type != MCAO_WFS_NGS && p.type != MCAO_WFS_LGS) return fail(S, MCAO_E_INVALID_ARG, "wfs %d: bad type", w);
        if (p.n_sub < 1 || p.n_px < 1 || p.n_fft < 1 || p.n_bin < 1)
            return fail(S, MCAO_E_INVALID_ARG, "wfs %d: sizes must be positive", w);
        if (p.n_fft < 2 * p.n_px) return fail(S, MCAO_E_UNSUPPORTED, "wfs %d: n_fft must be >= 2 n_px", w);
        if (p.n_fft % p.n_bin) return fail(S, MCAO_E_INVALID_ARG, "wfs %d: n_bin must divide n_fft", w);
        if ((long long)p.n_sub * p.n_px > 16384) return fail(S, MCAO_E_UNSUPPORTED, "wfs %d: pupil grid too large", w);
        if (!(is_fin(p.lambda) && p.lambda > 0)) return fail(S, MCAO_E_INVALID_ARG, "wfs %d: lambda must be > 0", w);
        if (!(is_fin(p.n_photons) && p.n_photons >= 0) || !(is_fin(p.read_noise) && p.read_noise >= 0))
            return fail(S, MCAO_E_INVALID_ARG, "wfs %d: flux and read noise must be >= 0", w);
        if (!(is_fin(p.valid_thr) && p.valid_thr >= 0 && p.valid_thr <= 1))
            return fail(S, MCAO_E_INVALID_ARG, "wfs %d: valid_thr must be in [0, 1]", w);
        if (!is_fin(p.theta_x) || !is_fin(p.theta_y) || !is_fin(p.launch_x) || !is_fin(p.launch_y))
            return fail(S, MCAO_E_INVALID_ARG, "wfs %d: non-finite direction or launch", w);
        if (p.type == MCAO_WFS_LGS && !(is_fin(p.height) && p.height > 0))
            return fail(S, MCAO_E_INVALID_ARG, "wfs %d: LGS height must be > 0", w);
        if (!(is_fin(p.na_fwhm) && p.na_fwhm >= 0)) return fail(S, MCAO_E_INVALID_ARG, "wfs %d: na_fwhm must be >= 0", w);
        bool el = p.type == MCAO_WFS_LGS && p.na_fwhm > 0;
        if (!wfs_variant_supported(p.n_px, p.n_fft, p.n_bin, el))
            return fail(S, MCAO_E_UNSUPPORTED, "wfs %d: no kernel for n_px=%d n_fft=%d n_bin=%d%s", w, p.n_px,
                        p.n_fft, p.n_bin, el ? " with elongation" : "");
    }
    for (int q = 0; q < c->n_sci; ++q) {
        const mcao_science& p = c->sci[q];
        if (p.n_px < 8 || p.n_px % 8 || p.pad < 1)
            return fail(S, MCAO_E_UNSUPPORTED, "science %d: n_px must be a multiple of 8, pad >= 1", q);
        if (!(is_fin(p.lambda) && p.lambda > 0)) return fail(S, MCAO_E_INVALID_ARG, "science %d: lambda must be > 0", q);
        if (!is_fin(p.theta_x) || !is_fin(p.theta_y))
            return fail(S, MCAO_E_INVALID_ARG, "science %d: non-finite direction", q);
        int M = p.n_px * p.pad;
        if (factor_fft(M).empty() || M > 4096)
            return fail(S, MCAO_E_UNSUPPORTED, "science %d: FFT size %d must factor into 2,3,5 and be <= 4096", q, M);
    }
    return MCAO_OK;
}

mcao_status d2h(mcao_sim* S, void* dst, const void* src, size_t bytes) {
    CK(cudaSetDevice(S->device));
    mcao_status r = sync_all(S);
    if (r != MCAO_OK) return r;
    if (bytes) CK(cudaMemcpy(dst, src, bytes, cudaMemcpyDeviceToHost));
    return MCAO_OK;
}

}  // namespace

// =============================================================================================
// C ABI
// =============================================================================================
extern "C" {

const char* mcao_create_error(void) { return g_create_error.c_str(); }

const char* mcao_last_error(const mcao_sim* sim) { return sim ? sim->err.c_str() : "null handle"; }

mcao_status mcao_sim_create(const mcao_config* cfg, mcao_sim** out) {
    g_create_error.clear();
    if (!out) return fail(nullptr, MCAO_E_INVALID_ARG, "out is NULL");
    *out = nullptr;
    mcao_status vs = validate_config(cfg);
    if (vs != MCAO_OK) return vs;
    mcao_sim* S = new mcao_sim();
    S->cfg = *cfg;
    S->cfg.wfs = nullptr;
    S->cfg.sci = nullptr;
    S->n_real = cfg->n_real;
    S->atm_loaded_r.assign(cfg->n_real, 0);
    auto bail = [&](mcao_status s) {
        g_create_error = S->err;
        destroy_all(S);
        return s;
    };
#define CKC(expr)                                                                                \
    do {                                                                                         \
        cudaError_t e_ = (expr);                                                                 \
        if (e_ != cudaSuccess) {                                                                 \
            fail(S, e_ == cudaErrorMemoryAllocation ? MCAO_E_OOM : MCAO_E_CUDA, "%s: %s", #expr,  \
                 cudaGetErrorString(e_));                                                        \
            return bail(e_ == cudaErrorMemoryAllocation ? MCAO_E_OOM : MCAO_E_CUDA);             \
        }                                                                                        \
    } while (0)
    CKC(cudaGetDevice(&S->device));
    CKC(cudaDeviceGetAttribute(&S->sm_count, cudaDevAttrMultiProcessorCount, S->device));
    int prio_lo = 0, prio_hi = 0;
    CKC(cudaDeviceGetStreamPriorityRange(&prio_lo, &prio_hi));
    // the reconstructor stream is served first so that its few resident blocks keep HBM busy
    // while the sensing kernels fill the remaining slots; science runs last
    CKC(cudaStreamCreateWithPriority(&S->s3, cudaStreamNonBlocking, prio_hi));
    CKC(cudaStreamCreateWithPriority(&S->s0, cudaStreamNonBlocking, (prio_lo + prio_hi) / 2));
    CKC(cudaStreamCreateWithPriority(&S->s1, cudaStreamNonBlocking, (prio_lo + prio_hi) / 2));
    CKC(cudaStreamCreateWithPriority(&S->s2, cudaStreamNonBlocking, prio_lo));
    CKC(cudaStreamCreateWithPriority(&S->s_read, cudaStreamNonBlocking, prio_lo));
    CKC(cudaEventCreateWithFlags(&S->ev_user, cudaEventDisableTiming));
    CKC(cudaEventCreateWithFlags(&S->ev_done, cudaEventDisableTiming));
    CKC(wfs_prepare());
    CKC(recon_prepare());
    CKC(multi_prepare());
    CKC(dalloc(&S->d_err, 1));
    CKC(cudaMemsetAsync(S->d_err, 0, sizeof(int), S->s0));
    CKC(dalloc(&S->d_work, (size_t)(2 * cfg->n_wfs + 1)));
    CKC(cudaMemsetAsync(S->d_work, 0, sizeof(unsigned int) * (2 * cfg->n_wfs + 1), S->s0));

    // ---- wavefront sensors
    int ns = 0, nframe = 0, ld = 0;
    std::vector<WfsDev> wdev;
    std::vector<float> amp_all;
    std::vector<size_t> amp_off;
    for (int w = 0; w < cfg->n_wfs; ++w) {
        WfsHost H;
        H.p = cfg->wfs[w];
        H.N = H.p.n_sub * H.p.n_px;
        H.dx = cfg->D / (double)H.N;
        H.n_det = H.p.n_fft / H.p.n_bin;
        H.fft_route = wfs_variant_is_fft(H.p.n_px, H.p.n_fft, H.p.n_bin);
        H.amp = pupil(cfg->D, cfg->obstruction, H.N);
        const int npx = H.p.n_px;
        for (int sy = 0; sy < H.p.n_sub; ++sy)
            for (int sx = 0; sx < H.p.n_sub; ++sx) {
                double s = 0.0;
                for (int y = 0; y < npx; ++y)
                    for (int x = 0; x < npx; ++x) s += H.amp[(size_t)(sy * npx + y) * H.N + sx * npx + x];
                double f = s / (double)(npx * npx);
                if (f >= H.p.valid_thr) {
                    H.valid.push_back(sy * H.p.n_sub + sx);
                    H.frac.push_back(f);
                }
            }
        H.n_valid = (int)H.valid.size();
        H.slope0 = ns;
        ns += 2 * H.n_valid;
        H.rcol0 = ld;
        ld += (2 * H.n_valid + 3) / 4 * 4;
        H.frame0 = nframe;
        nframe += H.n_valid * H.n_det * H.n_det;
        bool el = H.p.type == MCAO_WFS_LGS && H.p.na_fwhm > 0;
        for (int v = 0; v < H.n_valid; ++v) {
            SubapDev d{};
            d.wfs = w;
            d.sx = H.valid[v] % H.p.n_sub;
            d.sy = H.valid[v] / H.p.n_sub;
            d.rank = v;
            d.frac = (float)H.frac[v];
            if (el) set_elongation(H, d);
            H.subaps.push_back(d);
        }
        CKC(dalloc(&H.d_subaps, H.subaps.size()));
        if (!H.subaps.empty())
            CKC(cudaMemcpyAsync(H.d_subaps, H.subaps.data(), sizeof(SubapDev) * H.subaps.size(), cudaMemcpyHostToDevice, S->s0));
        WfsDev D{};
        D.type = H.p.type;
        D.n_sub = H.p.n_sub; D.n_px = npx; D.n_fft = H.p.n_fft; D.n_bin = H.p.n_bin; D.n_det = H.n_det;
        D.N = H.N;
        D.n_valid = H.n_valid; D.slope0 = H.slope0; D.frame0 = H.frame0; D.rcol0 = H.rcol0; D.wfs_index = w;
        D.scale = (float)(cfg->lambda_ref / H.p.lambda);
        D.n_photons = (float)H.p.n_photons;
        D.read_noise = (float)H.p.read_noise;
        for (int u = -(npx - 1); u <= npx - 1 && npx <= kMaxNpx; ++u) {
            double re = 0, im = 0;
            for (int t = 0; t < H.p.n_bin; ++t) {
                double a = 2.0 * M_PI * (double)u * t / (double)H.p.n_fft;
                re += std::cos(a);
                im += std::sin(a);
            }
            double sgn = (((u % 2) + 2) % 2) ? -1.0 : 1.0;
            D.h[u + npx - 1] = make_float2((float)(sgn * re), (float)(sgn * im));
        }
        for (int k = 0; k < H.n_det && k < kMaxNd; ++k) {
            double a = 2.0 * M_PI * (double)k / (double)H.n_det;
            D.tw[k] = make_float2((float)std::cos(a), (float)std::sin(a));
        }
        amp_off.push_back(amp_all.size());
        amp_all.insert(amp_all.end(), H.amp.begin(), H.amp.end());
        wdev.push_back(D);
        S->wfs.push_back(std::move(H));
    }
    S->n_slopes = ns;
    S->n_frame_px = nframe;
    S->ld = std::max(ld, 4);
    CKC(dalloc(&S->d_amp_all, amp_all.size()));
    CKC(cudaMemcpyAsync(S->d_amp_all, amp_all.data(), sizeof(float) * amp_all.size(), cudaMemcpyHostToDevice, S->s0));
    for (size_t w = 0; w < wdev.size(); ++w) wdev[w].amp = S->d_amp_all + amp_off[w];
    CKC(dalloc(&S->d_wfs, wdev.size()));
    CKC(cudaMemcpyAsync(S->d_wfs, wdev.data(), sizeof(WfsDev) * wdev.size(), cudaMemcpyHostToDevice, S->s0));
    const size_t NR = (size_t)S->n_real;
    CKC(dalloc(&S->d_slopes, NR * std::max(ns, 1)));
    CKC(cudaMemsetAsync(S->d_slopes, 0, sizeof(float) * NR * std::max(ns, 1), S->s0));
    CKC(dalloc(&S->d_slopes_pad, NR * pad_stride(S)));
    CKC(cudaMemsetAsync(S->d_slopes_pad, 0, sizeof(float) * NR * pad_stride(S), S->s0));
    CKC(dalloc(&S->d_sref, ns));
    CKC(cudaMemsetAsync(S->d_sref, 0, sizeof(float) * std::max(ns, 1), S->s0));
    if (cfg->keep_frames) {
        CKC(dalloc(&S->d_lam, NR * std::max(nframe, 1)));
        CKC(dalloc(&S->d_frames, NR * std::max(nframe, 1)));
        CKC(cudaMemsetAsync(S->d_lam, 0, sizeof(float) * NR * std::max(nframe, 1), S->s0));
        CKC(cudaMemsetAsync(S->d_frames, 0, sizeof(int) * NR * std::max(nframe, 1), S->s0));
    }

    // ---- block-per-subaperture sensors: one launch per kernel variant
    for (int w = 0; w < cfg->n_wfs; ++w) {
        if (!S->wfs[w].fft_route) continue;
        const mcao_wfs& p = cfg->wfs[w];
        FftGroup* g = nullptr;
        for (auto& x : S->fft_groups)
            if (x.n_px == p.n_px && x.n_fft == p.n_fft && x.n_bin == p.n_bin) g = &x;
        if (!g) {
            S->fft_groups.push_back(FftGroup{p.n_px, p.n_fft, p.n_bin, {}, nullptr, 0});
            g = &S->fft_groups.back();
        }
        g->wfs.push_back(w);
    }
    for (auto& g : S->fft_groups) {
        std::vector<SubapDev> all;
        for (int w : g.wfs) all.insert(all.end(), S->wfs[w].subaps.begin(), S->wfs[w].subaps.end());
        g.n_subaps = (int)all.size();
        CKC(dalloc(&g.d_subaps, all.size()));
        if (!all.empty())
            CKC(cudaMemcpyAsync(g.d_subaps, all.data(), sizeof(SubapDev) * all.size(), cudaMemcpyHostToDevice, S->s0));
    }

    // ---- science directions
    int maxM = 0;
    for (int q = 0; q < cfg->n_sci; ++q) {
        Science C;
        C.p = cfg->sci[q];
        C.N = C.p.n_px;
        C.M = C.p.n_px * C.p.pad;
        C.dx = cfg->D / (double)C.N;
        std::vector<float> A = pupil(cfg->D, cfg->obstruction, C.N);
        C.sum_amp = 0.0;
        for (float a : A) C.sum_amp += a;
        C.n_tiles = (C.N / 8) * (C.N / 8);
        C.radices = factor_fft(C.M);
        CKC(dalloc(&C.d_amp, A.size()));
        CKC(cudaMemcpyAsync(C.d_amp, A.data(), sizeof(float) * A.size(), cudaMemcpyHostToDevice, S->s0));
        CKC(dalloc(&C.d_field, NR * C.N * C.N));
        CKC(dalloc(&C.d_ft, NR * C.M * C.N));
        CKC(dalloc(&C.d_psf_t, NR * C.M * C.M));
        CKC(cudaMemsetAsync(C.d_psf_t, 0, sizeof(double) * NR * C.M * C.M, S->s0));
        CKC(dalloc(&C.d_sr_part, NR * std::max(C.n_tiles, 1)));
        const std::vector<float2> W = sci_twiddles(C.M);
        CKC(dalloc(&C.d_w, C.M));
        CKC(cudaMemcpyAsync(C.d_w, W.data(), sizeof(float2) * C.M, cudaMemcpyHostToDevice, S->s0));
        maxM = std::max(maxM, C.M);
        S->sci.push_back(C);
    }
    if (maxM > 0) {
        int dev_smem = 0;
        CKC(cudaDeviceGetAttribute(&dev_smem, cudaDevAttrMaxSharedMemoryPerBlockOptin, S->device));
        if (sci_smem_bytes(maxM) > (size_t)dev_smem) {
            fail(S, MCAO_E_UNSUPPORTED, "science FFT of %d points needs %zu B of shared memory", maxM,
                 sci_smem_bytes(maxM));
            return bail(MCAO_E_UNSUPPORTED);
        }
        CKC(sci_prepare(maxM));
    }
    CKC(dalloc(&S->d_acc, NR * std::max(cfg->n_sci, 1)));
    CKC(dalloc(&S->d_sr_out, 2 * (size_t)std::max(cfg->n_sci, 1)));
    CKC(cudaMemsetAsync(S->d_acc, 0, sizeof(SciAcc) * NR * std::max(cfg->n_sci, 1), S->s0));
    CKC(dalloc(&S->d_st, 1));
    CKC(cudaMemsetAsync(S->d_st, 0, sizeof(StepState), S->s0));
    CKC(cudaStreamSynchronize(S->s0));
    *out = S;
    return MCAO_OK;
#undef CKC
}

mcao_status mcao_sim_destroy(mcao_sim* sim) {
    destroy_all(sim);
    return MCAO_OK;
}

mcao_status mcao_set_stream(mcao_sim* S, void* stream) {
    if (!S) return MCAO_E_INVALID_ARG;
    S->user = (cudaStream_t)stream;
    S->user_set = true;
    return MCAO_OK;
}

mcao_status mcao_load_atmosphere(mcao_sim* S, int n_layers, const mcao_layer* layers) {
    if (!S) return MCAO_E_INVALID_ARG;
    if (n_layers < 0 || (n_layers > 0 && !layers)) return fail(S, MCAO_E_INVALID_ARG, "bad layer list");
    CK(cudaSetDevice(S->device));
    for (int l = 0; l < n_layers; ++l) {
        const mcao_layer& L = layers[l];
        if (L.n < 2 || L.n > kMaxGridN || !(is_fin(L.pixel_m) && L.pixel_m > 0) || !L.phase)
            return fail(S, MCAO_E_INVALID_ARG, "layer %d: 2 <= n <= %d, pixel > 0 and phase required", l, kMaxGridN);
        if (!is_fin(L.alt_m) || L.alt_m < 0 || !is_fin(L.vx) || !is_fin(L.vy))
            return fail(S, MCAO_E_INVALID_ARG, "layer %d: altitude and wind must be finite, altitude >= 0", l);
        for (const auto& w : S->wfs)
            if (w.p.type == MCAO_WFS_LGS && L.alt_m >= w.p.height)
                return fail(S, MCAO_E_INVALID_ARG, "layer %d lies above a laser guide star", l);
    }
    { mcao_status r_ = sync_all(S); if (r_ != MCAO_OK) return r_; }
    // every realization shares the layers' geometry; a different geometry (allowed for
    // realization 0 only) discards the screens of the other realizations
    bool same = n_layers == S->n_layers && (int)S->layers.size() == n_layers;
    for (int l = 0; same && l < n_layers; ++l) {
        const mcao_layer &a = layers[l], &b = S->layers[l];
        same = a.n == b.n && a.pixel_m == b.pixel_m && a.alt_m == b.alt_m && a.vx == b.vx && a.vy == b.vy;
    }
    if (!same) {
        if (S->cur != 0)
            return fail(S, MCAO_E_SHAPE, "realization %d: layers differ from realization 0's geometry", S->cur);
        for (auto p : S->d_layer_owned)
            if (p) cudaFree(p);
        S->d_layer_owned.assign((size_t)S->n_real * n_layers, nullptr);
        S->d_layer_ptr.assign((size_t)S->n_real * n_layers, nullptr);
        S->atm_loaded_r.assign(S->n_real, 0);
        S->layers.assign(layers, layers + n_layers);
        for (auto& L : S->layers) L.phase = nullptr;
        S->n_layers = n_layers;
    }
    S->atm_loaded = false;
    for (int l = 0; l < n_layers; ++l) {
        const mcao_layer& L = layers[l];
        const size_t slot = (size_t)S->cur * n_layers + l;
        if (S->d_layer_owned[slot]) {
            cudaFree(S->d_layer_owned[slot]);
            S->d_layer_owned[slot] = nullptr;
        }
        if (L.on_device) {
            S->d_layer_ptr[slot] = L.phase;
        } else {
            float* d = nullptr;
            CK(dalloc(&d, (size_t)L.n * L.n));
            S->d_layer_owned[slot] = d;
            CK(cudaMemcpyAsync(d, L.phase, sizeof(float) * (size_t)L.n * L.n, cudaMemcpyHostToDevice, S->s0));
            S->d_layer_ptr[slot] = d;
        }
    }
    S->atm_loaded_r[S->cur] = 1;
    mcao_status r = rebuild_views(S);
    if (r != MCAO_OK) return r;
    S->atm_loaded = std::all_of(S->atm_loaded_r.begin(), S->atm_loaded_r.end(), [](char c) { return c != 0; });
    CK(cudaStreamSynchronize(S->s0));
    return MCAO_OK;
}

// Gaussian tables Gx [surf_n][nx], Gy [surf_n][ny] of every DM (with its shift and
// magnification folded in: sample coordinate (x - shift) / mag), the per-tile actuator bands
// (weights >= 1e-10) and the misregistration fields of the descriptors.
static mcao_status build_dm_tables(mcao_sim* S, std::vector<float>& g, std::vector<int2>& band) {
    g.clear();
    band.clear();
    S->dm_nb = 1;
    for (int m = 0; m < S->n_dms; ++m) {
        const mcao_dm& d = S->dms[m];
        DmDesc& D = S->dm_desc[m];
        const std::array<double, 4>& T = S->dm_misreg[m];
        const double sig = d.pitch_m / std::sqrt(2.0 * std::log(1.0 / d.coupling));
        const double thr = 1e-10;
        auto table = [&](int na, double shift, long long& tband) {
            long long off = (long long)g.size();
            std::vector<int2> rows;
            for (int i = 0; i < d.surf_n; ++i) {
                double x = (((double)i - 0.5 * (double)(d.surf_n - 1)) * d.surf_dx - shift) / T[3];
                int lo = na, hi = 0;
                for (int a = 0; a < na; ++a) {
                    double xa = ((double)a - 0.5 * (double)(na - 1)) * d.pitch_m;
                    double v = std::exp(-(x - xa) * (x - xa) / (2.0 * sig * sig));
                    g.push_back((float)v);
                    if (v >= thr) { lo = std::min(lo, a); hi = std::max(hi, a + 1); }
                }
                rows.push_back(make_int2(lo, hi));
            }
            tband = (long long)band.size();
            for (int t = 0; t < D.tiles_x; ++t) {
                int lo = na, hi = 0;
                for (int i = t * kDmTile; i < std::min(d.surf_n, (t + 1) * kDmTile); ++i)
                    if (rows[i].y > rows[i].x) { lo = std::min(lo, rows[i].x); hi = std::max(hi, rows[i].y); }
                if (lo >= hi) { lo = 0; hi = 0; }
                band.push_back(make_int2(lo, hi));
            }
            return off;
        };
        D.general = T[2] != 0.0;
        // with rotation the tables describe the unrotated DM (kept for the band sizes only)
        D.gx_off = table(d.nx, D.general ? 0.0 : T[0], D.tband_x);
        D.gy_off = table(d.ny, D.general ? 0.0 : T[1], D.tband_y);
        // the same tables transposed ([actuator][sample]) for the forward kernel's staging
        auto transposed = [&](long long off, int na) {
            const long long toff = (long long)g.size();
            for (int a = 0; a < na; ++a)
                for (int i = 0; i < d.surf_n; ++i) {
                    const float v = g[off + (long long)i * na + a];
                    g.push_back(v);
                }
            return toff;
        };
        D.gxt_off = transposed(D.gx_off, d.nx);
        D.gyt_off = transposed(D.gy_off, d.ny);
        // block bands (union of two tiles' bands): the forward kernel's shared memory
        for (long long tb : {D.tband_x, D.tband_y})
            for (int t = 0; t < (D.tiles_x + 1) / 2; ++t) {
                const int2 a = band[tb + 2 * t];
                const int2 b = 2 * t + 1 < D.tiles_x ? band[tb + 2 * t + 1] : make_int2(0, 0);
                int w = std::max(a.y - a.x, b.y - b.x);
                if (a.y > a.x && b.y > b.x) w = std::max(a.y, b.y) - std::min(a.x, b.x);
                S->dm_nb = std::max(S->dm_nb, w);
            }
        if (!D.general)
            for (int t = 0; t < 2 * D.tiles_x; ++t) {
                int2 b = band[(t < D.tiles_x ? D.tband_x : D.tband_y) + t % D.tiles_x];
                if (b.y - b.x > kDmMaxBand)
                    return fail(S, MCAO_E_UNSUPPORTED, "dm %d: more than %d actuators per axis act on a %d-sample tile",
                                m, kDmMaxBand, kDmTile);
            }
        D.cr = (float)std::cos(T[2]);
        D.sr = (float)std::sin(T[2]);
        D.inv_mag = (float)(1.0 / T[3]);
        D.shx = (float)T[0];
        D.shy = (float)T[1];
        D.dx = (float)d.surf_dx;
        D.pitch = (float)d.pitch_m;
        D.inv2s2 = (float)(1.0 / (2.0 * sig * sig));
        D.rc = (float)(sig * std::sqrt(2.0 * std::log(1.0 / thr)) / d.pitch_m);
    }
    return MCAO_OK;
}

mcao_status mcao_set_misregistration(mcao_sim* S, int dm, double shift_x, double shift_y, double rotation,
                                     double magnification) {
    if (!S) return MCAO_E_INVALID_ARG;
    if (!S->dms_loaded) return fail(S, MCAO_E_STATE, "DMs not loaded");
    if (dm < 0 || dm >= S->n_dms) return fail(S, MCAO_E_INVALID_ARG, "bad DM index");
    if (!is_fin(shift_x) || !is_fin(shift_y) || !is_fin(rotation) || std::fabs(rotation) > M_PI ||
        !(is_fin(magnification) && magnification > 0.5 && magnification < 2.0))
        return fail(S, MCAO_E_INVALID_ARG, "finite shift, |rotation| <= pi and magnification in (0.5, 2) required");
    CK(cudaSetDevice(S->device));
    { mcao_status r_ = sync_all(S); if (r_ != MCAO_OK) return r_; }
    const std::array<double, 4> old = S->dm_misreg[dm];
    S->dm_misreg[dm] = {shift_x, shift_y, rotation, magnification};
    std::vector<float> g;
    std::vector<int2> band;
    mcao_status r = build_dm_tables(S, g, band);
    if (r != MCAO_OK) {
        S->dm_misreg[dm] = old;
        std::vector<float> g2;
        std::vector<int2> b2;
        build_dm_tables(S, g2, b2);
        return r;
    }
    release_graph(S);
    CK(dm_prepare());
    dfree(S->d_dm_g);
    dfree(S->d_dm_band);
    CK(dalloc(&S->d_dm_g, g.size()));
    CK(cudaMemcpyAsync(S->d_dm_g, g.data(), sizeof(float) * g.size(), cudaMemcpyHostToDevice, S->s0));
    CK(dalloc(&S->d_dm_band, band.size()));
    CK(cudaMemcpyAsync(S->d_dm_band, band.data(), sizeof(int2) * band.size(), cudaMemcpyHostToDevice, S->s0));
    CK(cudaMemcpyAsync(S->d_dm_desc, S->dm_desc.data(), sizeof(DmDesc) * S->n_dms, cudaMemcpyHostToDevice, S->s0));
    CK(cudaStreamSynchronize(S->s0));
    return MCAO_OK;
}

mcao_status mcao_load_dms(mcao_sim* S, int n_dms, const mcao_dm* dms) {
    if (!S) return MCAO_E_INVALID_ARG;
    if (n_dms < 0 || n_dms > kMaxDms || (n_dms > 0 && !dms))
        return fail(S, MCAO_E_INVALID_ARG, "n_dms must be in [0, %d]", kMaxDms);
    for (int m = 0; m < n_dms; ++m) {
        const mcao_dm& d = dms[m];
        if (d.nx < 1 || d.ny < 1 || !d.valid || d.surf_n < 2 || !(is_fin(d.surf_dx) && d.surf_dx > 0) ||
            !(is_fin(d.pitch_m) && d.pitch_m > 0) || !(is_fin(d.coupling) && d.coupling > 0 && d.coupling < 1) ||
            !is_fin(d.alt_m) || d.alt_m < 0)
            return fail(S, MCAO_E_INVALID_ARG, "dm %d: invalid geometry", m);
        if (d.surf_n > kMaxGridN)
            return fail(S, MCAO_E_UNSUPPORTED, "dm %d: at most %d surface samples per side", m, kMaxGridN);
        for (const auto& w : S->wfs)
            if (w.p.type == MCAO_WFS_LGS && d.alt_m >= w.p.height)
                return fail(S, MCAO_E_INVALID_ARG, "dm %d lies above a laser guide star", m);
    }
    CK(cudaSetDevice(S->device));
    { mcao_status r_ = sync_all(S); if (r_ != MCAO_OK) return r_; }
    dfree(S->d_dm_desc); dfree(S->d_dm_g); dfree(S->d_dm_band); dfree(S->d_dm_map);
    dfree(S->d_dm_surf); dfree(S->d_c); dfree(S->d_partial);
    S->dms_loaded = false;
    S->recon_loaded = false;  // command count may change
    S->dms.assign(dms, dms + n_dms);
    S->n_dms = n_dms;
    S->dm_desc.clear();
    S->dm_cmd0.assign(n_dms + 1, 0);
    std::vector<float> g;
    std::vector<int2> band;
    std::vector<int> map;
    long long surf_total = 0;
    int ncmd = 0, tiles = 0;
    for (int m = 0; m < n_dms; ++m) {
        const mcao_dm& d = dms[m];
        DmDesc D{};
        D.nx = d.nx; D.ny = d.ny; D.surf_n = d.surf_n;
        D.tiles_x = (d.surf_n + kDmTile - 1) / kDmTile;
        D.map_off = (long long)map.size();
        int cnt = 0;
        for (int a = 0; a < d.nx * d.ny; ++a) {
            if (d.valid[a]) { map.push_back(ncmd + cnt); ++cnt; }
            else map.push_back(-1);
        }
        ncmd += cnt;
        S->dm_cmd0[m + 1] = ncmd;
        D.surf_off = surf_total;
        surf_total += (long long)d.surf_n * d.surf_n;
        S->dm_tile_start[m] = tiles;
        tiles += ((D.tiles_x + 1) / 2) * ((D.tiles_x + 1) / 2);   // 64 x 64 blocks
        S->dm_desc.push_back(D);
    }
    for (int m = n_dms; m <= kMaxDms; ++m) S->dm_tile_start[m] = tiles;
    S->n_cmd = ncmd;
    S->dm_misreg.assign(n_dms, {0.0, 0.0, 0.0, 1.0});
    { mcao_status r_ = build_dm_tables(S, g, band); if (r_ != MCAO_OK) return r_; }
    CK(dm_prepare());
    CK(dalloc(&S->d_dm_desc, S->dm_desc.size()));
    if (n_dms) CK(cudaMemcpyAsync(S->d_dm_desc, S->dm_desc.data(), sizeof(DmDesc) * n_dms, cudaMemcpyHostToDevice, S->s0));
    CK(dalloc(&S->d_dm_g, g.size()));
    if (!g.empty()) CK(cudaMemcpyAsync(S->d_dm_g, g.data(), sizeof(float) * g.size(), cudaMemcpyHostToDevice, S->s0));
    CK(dalloc(&S->d_dm_band, band.size()));
    if (!band.empty()) CK(cudaMemcpyAsync(S->d_dm_band, band.data(), sizeof(int2) * band.size(), cudaMemcpyHostToDevice, S->s0));
    CK(dalloc(&S->d_dm_map, map.size()));
    if (!map.empty()) CK(cudaMemcpyAsync(S->d_dm_map, map.data(), sizeof(int) * map.size(), cudaMemcpyHostToDevice, S->s0));
    S->surf_total = surf_total;
    CK(dalloc(&S->d_dm_surf, (size_t)S->n_real * std::max<long long>(surf_total, 1)));
    CK(cudaMemsetAsync(S->d_dm_surf, 0, sizeof(float) * (size_t)S->n_real * std::max<long long>(surf_total, 1), S->s0));
    CK(dalloc(&S->d_c, (size_t)S->n_real * std::max(ncmd, 1)));
    CK(cudaMemsetAsync(S->d_c, 0, sizeof(float) * (size_t)S->n_real * std::max(ncmd, 1), S->s0));
    for (float** p : {&S->d_c_prev, &S->d_dc_prev, &S->d_dc}) {
        dfree(*p);
        CK(dalloc(p, (size_t)S->n_real * std::max(ncmd, 1)));
        CK(cudaMemsetAsync(*p, 0, sizeof(float) * (size_t)S->n_real * std::max(ncmd, 1), S->s0));
    }
    mcao_status r = rebuild_views(S);
    if (r != MCAO_OK) return r;
    S->dms_loaded = true;
    CK(cudaStreamSynchronize(S->s0));
    return MCAO_OK;
}

mcao_status mcao_load_reconstructor(mcao_sim* S, int n_cmd, int n_slopes, const float* R, const float* s_ref,
                                    int dtype, int on_device) {
    if (!S) return MCAO_E_INVALID_ARG;
    if (!S->dms_loaded) return fail(S, MCAO_E_STATE, "load the DMs before the reconstructor");
    if (dtype != MCAO_DTYPE_F32 && dtype != MCAO_DTYPE_BF16 && dtype != MCAO_DTYPE_FP8_E4M3)
        return fail(S, MCAO_E_UNSUPPORTED, "unknown reconstructor dtype %d", dtype);
    if (n_cmd != S->n_cmd || n_slopes != S->n_slopes)
        return fail(S, MCAO_E_SHAPE, "reconstructor is %d x %d, configuration needs %d x %d", n_cmd, n_slopes,
                    S->n_cmd, S->n_slopes);
    if (!R && n_cmd > 0) return fail(S, MCAO_E_INVALID_ARG, "R is NULL");
    if (n_slopes < 1) return fail(S, MCAO_E_SHAPE, "no valid subapertures");
    CK(cudaSetDevice(S->device));
    { mcao_status r_ = sync_all(S); if (r_ != MCAO_OK) return r_; }
    dfree(S->d_R);
    dfree(S->d_rscale);
    dfree(S->d_partial);
    S->r_dtype = dtype;
    S->recon_loaded = false;
    S->rows_pad = std::max(1, (n_cmd + kReconRowBlock - 1) / kReconRowBlock) * kReconRowBlock;
    const cudaMemcpyKind kind = on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice;
    // device inputs may come from any stream of the caller: wait for all of them
    if (on_device) CK(cudaDeviceSynchronize());
    // 1) row-major staging copy in the padded column layout (each sensor's slope block starts on
    //    a 16-byte boundary of a row, rows padded with zeros)
    float* tmp = nullptr;
    size_t elems = (size_t)S->rows_pad * S->ld;
    CK(dalloc(&tmp, elems));
    cudaError_t e = cudaMemsetAsync(tmp, 0, sizeof(float) * elems, S->s0);
    // 2) slices.  Block-per-subaperture sensors first (their kernel runs beside the first
    //    warp-per-subaperture sensor, so their slice can run before that sensor is done), and
    //    runs of them adjacent in the padded layout merged into one slice; then one slice per
    //    warp-per-subaperture sensor, in sensor order.
    S->slices.clear();
    S->slice_wfs.clear();
    int chunks = 0;
    long long tiled = 0;
    for (size_t w = 0; w < S->wfs.size(); ++w) {
        const WfsHost& W = S->wfs[w];
        const int len = 2 * W.n_valid;
        if (len > 0 && e == cudaSuccess && n_cmd > 0)
            e = cudaMemcpy2DAsync(tmp + W.rcol0, sizeof(float) * S->ld, R + W.slope0, sizeof(float) * n_slopes,
                                  sizeof(float) * len, n_cmd, kind, S->s0);
    }
    if (S->n_real > 1) {
        // batched product: float32 R column-major for the CUDA-core product, or the tensor-core
        // product's bfloat16 copy
        dfree(S->d_Rrm);
        dfree(S->d_multi_st);
        dfree(S->d_multi_part);
        S->d_Rrm = S->d_multi_st = S->d_multi_part = nullptr;
        tc_destroy(S->tc);
        S->tc = nullptr;
        if (dtype == MCAO_DTYPE_F32) {
            // column-major [ld][rows_pad] (streamed column by column), scratch for kMultiRhs
            // realizations per pass
            if (e == cudaSuccess) e = dalloc(&S->d_Rrm, elems);
            if (e == cudaSuccess) e = launch_transpose(tmp, S->rows_pad, S->ld, S->d_Rrm, S->rows_pad, 0, S->s0);
            if (e == cudaSuccess) e = dalloc(&S->d_multi_st, (size_t)S->ld * kMultiRhs);
            if (e == cudaSuccess)
                e = dalloc(&S->d_multi_part, (size_t)multi_chunks(S->ld) * kMultiRhs * std::max(n_cmd, 1));
        } else if (e == cudaSuccess && n_cmd > 0) {
            e = tc_create(tmp, S->rows_pad, S->ld, n_cmd, S->n_real, S->sm_count, dtype == MCAO_DTYPE_FP8_E4M3 ? 1 : 0,
                          S->s0, &S->tc);
        }
        if (e == cudaSuccess) e = cudaStreamSynchronize(S->s0);
        cudaFree(tmp);
        CK(e);
        S->n_chunks = 0;
        CK(dalloc(&S->d_partial, 1));
        if (s_ref)
            CK(cudaMemcpyAsync(S->d_sref, s_ref, sizeof(float) * n_slopes, kind, S->s0));
        else
            CK(cudaMemsetAsync(S->d_sref, 0, sizeof(float) * n_slopes, S->s0));
        CK(cudaStreamSynchronize(S->s0));
        release_graph(S);
        S->recon_loaded = true;
        return MCAO_OK;
    }
    std::vector<std::vector<int>> units;
    for (const auto& g : S->fft_groups) {
        std::vector<int> ws;
        for (int w : g.wfs)
            if (S->wfs[w].n_valid > 0) ws.push_back(w);
        std::sort(ws.begin(), ws.end(), [&](int a, int b) { return S->wfs[a].rcol0 < S->wfs[b].rcol0; });
        for (int w : ws) {
            if (!units.empty()) {
                const WfsHost& P = S->wfs[units.back().back()];
                const bool same_group = std::find(g.wfs.begin(), g.wfs.end(), units.back().back()) != g.wfs.end();
                if (same_group && S->wfs[w].rcol0 == P.rcol0 + (2 * P.n_valid + 3) / 4 * 4) {
                    units.back().push_back(w);
                    continue;
                }
            }
            units.push_back({w});
        }
    }
    for (size_t w = 0; w < S->wfs.size(); ++w)
        if (!S->wfs[w].fft_route && S->wfs[w].n_valid > 0) units.push_back({(int)w});
    for (const auto& u : units) {
        const WfsHost& F = S->wfs[u.front()];
        const WfsHost& B = S->wfs[u.back()];
        const int len = B.rcol0 + 2 * B.n_valid - F.rcol0;
        ReconLaunch L{};
        L.n_cmd = n_cmd;
        L.n_rq = S->rows_pad / kReconRows;
        L.col0 = F.rcol0;
        L.len = len;
        // chunk width: at most kReconChunk columns, a multiple of 16, and (trying up to 8 more
        // chunks) such that each chunk's last stage holds 0 or at least half a stage of vectors
        const int epv = 16 / recon_esize(dtype);
        int nch = (len + kReconChunk - 1) / kReconChunk;
        auto chunk_cols = [&](int n) { return ((len + n - 1) / n + 15) / 16 * 16; };
        auto ok = [&](int w) {
            const int rem_full = (w / epv) % kReconSeg;
            const int last = len - (len + w - 1) / w * w + w;
            const int rem_last = ((last + epv - 1) / epv) % kReconSeg;
            return (rem_full == 0 || rem_full >= kReconSeg / 2) && (rem_last == 0 || rem_last >= kReconSeg / 2);
        };
        for (int extra = 0; extra <= 8; ++extra)
            if (ok(chunk_cols(nch + extra))) {
                nch += extra;
                break;
            }
        L.kc = chunk_cols(nch);
        nch = (len + L.kc - 1) / L.kc;
        L.dtype = dtype;
        L.chunk0 = chunks;
        L.base = tiled;
        L.s = S->d_slopes_pad;
        L.max_ctas = S->sm_count;  // one resident block per SM beside the sensing kernels
        L.err = S->d_err;
        chunks += nch;
        tiled += recon_slice_bytes(L.n_rq, L.len, L.kc, dtype);
        S->slices.push_back(L);
        S->slice_wfs.push_back(u);
    }
    for (size_t i = 0; i < S->slices.size(); ++i) S->slices[i].work = S->d_work + S->wfs.size() + i;
    // 3) stage-tiled copy used by the product (see ReconLaunch)
    if (e == cudaSuccess) e = dalloc(&S->d_R, (size_t)std::max<long long>(tiled, 16));
    if (e == cudaSuccess) e = cudaMemsetAsync(S->d_R, 0, (size_t)std::max<long long>(tiled, 16), S->s0);
    if (e == cudaSuccess && dtype == MCAO_DTYPE_FP8_E4M3) {
        e = dalloc(&S->d_rscale, (size_t)S->rows_pad);
        if (e == cudaSuccess) e = launch_recon_scales(tmp, S->rows_pad, S->ld, S->ld, S->d_rscale, S->s0);
    }
    for (auto& L : S->slices) {
        L.R = S->d_R;
        L.scale = S->d_rscale;
        if (e == cudaSuccess) e = launch_recon_tile(tmp, S->ld, L, S->s0);
    }
    if (e == cudaSuccess) e = cudaStreamSynchronize(S->s0);
    cudaFree(tmp);
    CK(e);
    S->n_chunks = chunks;
    CK(dalloc(&S->d_partial, (size_t)std::max(chunks, 1) * std::max(n_cmd, 1)));
    for (auto& L : S->slices) L.partial = S->d_partial;
    if (s_ref)
        CK(cudaMemcpyAsync(S->d_sref, s_ref, sizeof(float) * n_slopes, kind, S->s0));
    else
        CK(cudaMemsetAsync(S->d_sref, 0, sizeof(float) * n_slopes, S->s0));
    release_graph(S);
    S->recon_loaded = true;
    return MCAO_OK;
}

mcao_status mcao_step(mcao_sim* S, int n_steps) {
    if (!S) return MCAO_E_INVALID_ARG;
    if (n_steps < 0) return fail(S, MCAO_E_INVALID_ARG, "n_steps must be >= 0");
    if (!S->atm_loaded || !S->dms_loaded || !S->recon_loaded)
        return fail(S, MCAO_E_STATE, "load the atmosphere, the DMs and the reconstructor before stepping");
    if (n_steps == 0) return MCAO_OK;
    CK(cudaSetDevice(S->device));
    if (S->graph_dirty || S->graph_mask != S->prof_mask) {
        mcao_status r = build_graph(S);
        if (r != MCAO_OK) return r;
    }
    mcao_status r = order_after_user(S);
    if (r != MCAO_OK) return r;
    int i = 0;
    if (S->graph_k_steps > 1)
        for (; i + S->graph_k_steps <= n_steps; i += S->graph_k_steps) CK(cudaGraphLaunch(S->exec_k, S->s0));
    for (; i < n_steps; ++i) {
        if (S->profiling) {
            S->prof_step_begin.push_back(S->prof_records.size());
            for (const auto& p : S->prof_slots) {
                if (!p.na || !p.nb) continue;
                if (S->prof_used + 2 > S->prof_pool.size()) {
                    cudaEvent_t a, b;
                    CK(cudaEventCreate(&a));
                    CK(cudaEventCreate(&b));
                    S->prof_pool.push_back(a);
                    S->prof_pool.push_back(b);
                }
                cudaEvent_t ea = S->prof_pool[S->prof_used], eb = S->prof_pool[S->prof_used + 1];
                S->prof_used += 2;
                CK(cudaGraphExecEventRecordNodeSetEvent(S->exec, p.na, ea));
                CK(cudaGraphExecEventRecordNodeSetEvent(S->exec, p.nb, eb));
                S->prof_records.push_back({p.stage, {ea, eb}});
            }
        }
        CK(cudaGraphLaunch(S->exec, S->s0));
    }
    return signal_user(S);
}

mcao_status mcao_step_group(mcao_sim* const* sims, int n_sims, int n_steps) {
    if (!sims || n_sims < 1 || n_steps < 0) return MCAO_E_INVALID_ARG;
    for (int i = 0; i < n_sims; ++i) {
        mcao_sim* S = sims[i];
        if (!S) return MCAO_E_INVALID_ARG;
        for (int j = 0; j < i; ++j)
            if (sims[j] == S) return fail(S, MCAO_E_INVALID_ARG, "a simulation appears twice in the group");
        if (!S->atm_loaded || !S->dms_loaded || !S->recon_loaded)
            return fail(S, MCAO_E_STATE, "load the atmosphere, the DMs and the reconstructor before stepping");
        if (S->profiling) return fail(S, MCAO_E_UNSUPPORTED, "group steps run without the stage profiler");
        if (S->device != sims[0]->device) return fail(S, MCAO_E_INVALID_ARG, "the group spans devices");
    }
    if (n_steps == 0) return MCAO_OK;
    mcao_sim* S = sims[0];   // its s0 carries the group launches
    CK(cudaSetDevice(S->device));
    for (int i = 0; i < n_sims; ++i) {
        if (sims[i]->graph_dirty || sims[i]->graph_mask) {
            mcao_status r = build_graph(sims[i]);
            if (r != MCAO_OK) return r;
        }
        mcao_status r = order_after_user(sims[i]);
        if (r != MCAO_OK) return r;
    }
    // one parent graph: every simulation's step as an independent child
    cudaGraph_t parent = nullptr;
    cudaGraphExec_t exec = nullptr;
    cudaError_t e = cudaGraphCreate(&parent, 0);
    for (int i = 0; i < n_sims && e == cudaSuccess; ++i) {
        cudaGraphNode_t node;
        e = cudaGraphAddChildGraphNode(&node, parent, nullptr, 0, sims[i]->graph);
    }
    if (e == cudaSuccess) e = cudaGraphInstantiate(&exec, parent, cudaGraphInstantiateFlagUseNodePriority);
    // order after each simulation's earlier work, and each simulation's later work after the group
    for (int i = 1; i < n_sims && e == cudaSuccess; ++i) {
        e = cudaEventRecord(sims[i]->ev_done, sims[i]->s0);
        if (e == cudaSuccess) e = cudaStreamWaitEvent(S->s0, sims[i]->ev_done, 0);
    }
    for (int k = 0; k < n_steps && e == cudaSuccess; ++k) e = cudaGraphLaunch(exec, S->s0);
    if (e == cudaSuccess) e = cudaEventRecord(S->ev_done, S->s0);
    for (int i = 1; i < n_sims && e == cudaSuccess; ++i) e = cudaStreamWaitEvent(sims[i]->s0, S->ev_done, 0);
    if (exec) cudaGraphExecDestroy(exec);   // released once the queued launches complete
    if (parent) cudaGraphDestroy(parent);
    CK(e);
    for (int i = 0; i < n_sims; ++i) {
        mcao_status r = signal_user(sims[i]);
        if (r != MCAO_OK) return r;
    }
    return MCAO_OK;
}

mcao_status mcao_sync(mcao_sim* S) {
    if (!S) return MCAO_E_INVALID_ARG;
    CK(cudaSetDevice(S->device));
    return sync_all(S);
}

mcao_status mcao_query(const mcao_sim* S, int kind, int index, size_t* n) {
    if (!S || !n) return MCAO_E_INVALID_ARG;
    mcao_sim* Sm = const_cast<mcao_sim*>(S);
    switch (kind) {
        case MCAO_Q_SLOPES: *n = (size_t)S->n_slopes; return MCAO_OK;
        case MCAO_Q_COMMANDS:
            if (!S->dms_loaded) return fail(Sm, MCAO_E_STATE, "DMs not loaded");
            *n = (size_t)S->n_cmd;
            return MCAO_OK;
        case MCAO_Q_VALID:
        case MCAO_Q_FRAME:
        case MCAO_Q_WFS_PHASE:
            if (index < 0 || index >= (int)S->wfs.size()) return fail(Sm, MCAO_E_INVALID_ARG, "bad WFS index");
            if (kind == MCAO_Q_VALID) *n = (size_t)S->wfs[index].n_valid;
            else if (kind == MCAO_Q_FRAME) *n = (size_t)S->wfs[index].n_valid * S->wfs[index].n_det * S->wfs[index].n_det;
            else *n = (size_t)S->wfs[index].N * S->wfs[index].N;
            return MCAO_OK;
        case MCAO_Q_DM_SURFACE:
            if (index < 0 || index >= S->n_dms) return fail(Sm, MCAO_E_INVALID_ARG, "bad DM index");
            *n = (size_t)S->dms[index].surf_n * S->dms[index].surf_n;
            return MCAO_OK;
        case MCAO_Q_PSF:
            if (index < 0 || index >= (int)S->sci.size()) return fail(Sm, MCAO_E_INVALID_ARG, "bad science index");
            *n = (size_t)S->sci[index].M * S->sci[index].M;
            return MCAO_OK;
        case MCAO_Q_STATE: {
            size_t per = sizeof(float) * (3 * (size_t)S->n_cmd + S->n_slopes);
            for (const auto& c : S->sci) per += sizeof(SciAcc) + sizeof(double) * (size_t)c.M * c.M;
            *n = 4 * sizeof(int64_t) + per * (size_t)S->n_real;
            return MCAO_OK;
        }
        case MCAO_Q_REALIZATIONS: *n = (size_t)S->n_real; return MCAO_OK;
        default: return fail(Sm, MCAO_E_INVALID_ARG, "unknown query kind %d", kind);
    }
}

mcao_status mcao_get_step_index(mcao_sim* S, int64_t* k) {
    if (!S || !k) return MCAO_E_INVALID_ARG;
    StepState st;
    mcao_status r = d2h(S, &st, S->d_st, sizeof(st));
    if (r != MCAO_OK) return r;
    *k = st.k_next;
    return MCAO_OK;
}

mcao_status mcao_get_slopes(mcao_sim* S, float* out, size_t n) {
    if (!S || !out) return MCAO_E_INVALID_ARG;
    if (n < (size_t)S->n_slopes) return fail(S, MCAO_E_SHAPE, "need %d slopes", S->n_slopes);
    return d2h(S, out, S->d_slopes + (size_t)S->cur * S->n_slopes, sizeof(float) * S->n_slopes);
}

mcao_status mcao_get_commands(mcao_sim* S, float* out, size_t n) {
    if (!S || !out) return MCAO_E_INVALID_ARG;
    if (!S->dms_loaded) return fail(S, MCAO_E_STATE, "DMs not loaded");
    if (n < (size_t)S->n_cmd) return fail(S, MCAO_E_SHAPE, "need %d commands", S->n_cmd);
    return d2h(S, out, S->d_c + (size_t)S->cur * S->n_cmd, sizeof(float) * S->n_cmd);
}

mcao_status mcao_set_commands(mcao_sim* S, const float* in, size_t n) {
    if (!S || !in) return MCAO_E_INVALID_ARG;
    if (!S->dms_loaded) return fail(S, MCAO_E_STATE, "DMs not loaded");
    if (n != (size_t)S->n_cmd) return fail(S, MCAO_E_SHAPE, "need exactly %d commands", S->n_cmd);
    for (size_t i = 0; i < n; ++i)
        if (!std::isfinite(in[i])) return fail(S, MCAO_E_INVALID_ARG, "command %zu is not finite", i);
    CK(cudaSetDevice(S->device));
    { mcao_status r_ = sync_all(S); if (r_ != MCAO_OK) return r_; }
    if (n) {
        const size_t off = (size_t)S->cur * S->n_cmd;
        CK(cudaMemcpyAsync(S->d_c + off, in, sizeof(float) * n, cudaMemcpyHostToDevice, S->s0));
        CK(cudaMemcpyAsync(S->d_c_prev + off, in, sizeof(float) * n, cudaMemcpyHostToDevice, S->s0));
        CK(cudaMemsetAsync(S->d_dc_prev + off, 0, sizeof(float) * n, S->s0));
    }
    CK(cudaStreamSynchronize(S->s0));
    return MCAO_OK;
}

mcao_status mcao_get_valid(mcao_sim* S, int wfs, int32_t* out, size_t n) {
    if (!S || !out) return MCAO_E_INVALID_ARG;
    if (wfs < 0 || wfs >= (int)S->wfs.size()) return fail(S, MCAO_E_INVALID_ARG, "bad WFS index");
    const auto& v = S->wfs[wfs].valid;
    if (n < v.size()) return fail(S, MCAO_E_SHAPE, "need %zu entries", v.size());
    for (size_t i = 0; i < v.size(); ++i) out[i] = v[i];
    return MCAO_OK;
}

mcao_status mcao_get_wfs_phase(mcao_sim* S, int wfs, float* out, size_t n) {
    if (!S || !out) return MCAO_E_INVALID_ARG;
    if (wfs < 0 || wfs >= (int)S->wfs.size()) return fail(S, MCAO_E_INVALID_ARG, "bad WFS index");
    if (!S->atm_loaded || !S->dms_loaded) return fail(S, MCAO_E_STATE, "atmosphere and DMs must be loaded");
    const int N = S->wfs[wfs].N;
    if (n < (size_t)N * N) return fail(S, MCAO_E_SHAPE, "need %d samples", N * N);
    CK(cudaSetDevice(S->device));
    { mcao_status r_ = sync_all(S); if (r_ != MCAO_OK) return r_; }
    float* d = nullptr;
    CK(dalloc(&d, (size_t)N * N));
    cudaError_t e = launch_dm_surfaces(make_dm_launch(S), S->s0);
    if (e == cudaSuccess) e = launch_wfs_phase(make_ctx(S), S->cur, wfs, N, d, S->s0);
    if (e == cudaSuccess) e = cudaStreamSynchronize(S->s0);
    if (e == cudaSuccess) e = cudaMemcpy(out, d, sizeof(float) * (size_t)N * N, cudaMemcpyDeviceToHost);
    cudaFree(d);
    CK(e);
    return MCAO_OK;
}

// DM surfaces and every sensor at the current step and commands (no reconstruction, no time
// advance); noise as given
static cudaError_t enqueue_sensing(mcao_sim* S, int noise) {
    cudaError_t e = launch_dm_surfaces(make_dm_launch(S), S->s0);
    if (e != cudaSuccess) return e;
    auto run = [&](const SubapDev* sub, int n, unsigned int* work, int npx, int nfft, int nbin) {
        WfsLaunch L = make_wfs_launch(S, sub, n, work);
        L.ctx.noise = noise;
        if (!noise) L.frame_out = nullptr;
        return launch_wfs(L, npx, nfft, nbin, S->s0);
    };
    for (const auto& g : S->fft_groups)
        if ((e = run(g.d_subaps, g.n_subaps, nullptr, g.n_px, g.n_fft, g.n_bin)) != cudaSuccess) return e;
    for (size_t w = 0; w < S->wfs.size(); ++w) {
        const WfsHost& W = S->wfs[w];
        if (W.fft_route || W.n_valid == 0) continue;
        if ((e = run(W.d_subaps, W.n_valid, S->d_work + w, W.p.n_px, W.p.n_fft, W.p.n_bin)) != cudaSuccess) return e;
    }
    return cudaSuccess;
}

mcao_status mcao_measure(mcao_sim* S, int with_noise) {
    if (!S) return MCAO_E_INVALID_ARG;
    if (!S->atm_loaded || !S->dms_loaded) return fail(S, MCAO_E_STATE, "atmosphere and DMs must be loaded");
    CK(cudaSetDevice(S->device));
    { mcao_status r_ = sync_all(S); if (r_ != MCAO_OK) return r_; }
    CK(enqueue_sensing(S, with_noise ? S->cfg.noise : 0));
    CK(cudaStreamSynchronize(S->s0));
    return MCAO_OK;
}

mcao_status mcao_reconstruct_batch(mcao_sim* S, const float* slopes, int n_rhs, float* out) {
    if (!S) return MCAO_E_INVALID_ARG;
    if (!S->recon_loaded) return fail(S, MCAO_E_STATE, "load the reconstructor first");
    if (S->n_real < 2) return fail(S, MCAO_E_UNSUPPORTED, "the batched product needs n_real > 1");
    if (!slopes || !out) return fail(S, MCAO_E_INVALID_ARG, "slopes and out must be device pointers");
    if (n_rhs < 1 || n_rhs > S->n_real) return fail(S, MCAO_E_SHAPE, "n_rhs must be in [1, %d]", S->n_real);
    CK(cudaSetDevice(S->device));
    CK(cudaDeviceSynchronize());   // inputs produced on any stream are complete
    { mcao_status r_ = sync_all(S); if (r_ != MCAO_OK) return r_; }
    // the user layout [n_rhs][n_slopes] scattered into the padded layout of the product
    const int ps = pad_stride(S);
    CK(cudaMemsetAsync(S->d_slopes_pad, 0, sizeof(float) * (size_t)n_rhs * ps, S->s0));
    for (const WfsHost& W : S->wfs)
        if (W.n_valid > 0)
            CK(cudaMemcpy2DAsync(S->d_slopes_pad + W.rcol0, sizeof(float) * ps, slopes + W.slope0,
                                 sizeof(float) * S->n_slopes, sizeof(float) * 2 * W.n_valid, n_rhs,
                                 cudaMemcpyDeviceToDevice, S->s0));
    int nl = 0;
    CK(enqueue_batched_product(S, n_rhs, 1.0f, 0.0f, out, &nl));
    return sync_all(S);
}

// d slope / d phase of every slope on its subaperture's samples (current realization), then the
// command rows (D) or the command gradients (gvec -> gc) and the phase gradients
static mcao_status run_adjoint(mcao_sim* S, float* D, long long ld, const float* gvec, int n_vec, float* gc,
                               float* g_phase, float* g_layers) {
    int P = 1;
    for (const auto& W : S->wfs) P = std::max(P, W.p.n_px * W.p.n_px);
    CK(cudaDeviceSynchronize());   // inputs produced on any stream are complete
    { mcao_status r_ = sync_all(S); if (r_ != MCAO_OK) return r_; }
    float* sens = nullptr;
    int* d_err = nullptr;
    cudaError_t e = dalloc(&sens, (size_t)S->n_slopes * P);
    if (e == cudaSuccess) e = dalloc(&d_err, 1);
    if (e == cudaSuccess) e = cudaMemsetAsync(d_err, 0, sizeof(int), S->s0);
    if (e == cudaSuccess) e = launch_dm_surfaces(make_dm_launch(S), S->s0);
    long long phase_total = 0;
    for (const auto& W : S->wfs) phase_total += (long long)W.N * W.N;
    if (e == cudaSuccess && D) e = cudaMemsetAsync(D, 0, sizeof(float) * (size_t)S->n_slopes * ld, S->s0);
    if (e == cudaSuccess && gc) e = cudaMemsetAsync(gc, 0, sizeof(float) * (size_t)n_vec * S->n_cmd, S->s0);
    if (e == cudaSuccess && g_phase) e = cudaMemsetAsync(g_phase, 0, sizeof(float) * (size_t)n_vec * phase_total, S->s0);
    // layers concatenated: offsets and total length
    std::vector<long long> loff(S->n_layers + 1, 0);
    for (int l = 0; l < S->n_layers; ++l) loff[l + 1] = loff[l] + (long long)S->layers[l].n * S->layers[l].n;
    long long* d_loff = nullptr;
    if (e == cudaSuccess && g_layers) {
        e = cudaMemsetAsync(g_layers, 0, sizeof(float) * (size_t)n_vec * loff[S->n_layers], S->s0);
        if (e == cudaSuccess) e = dalloc(&d_loff, loff.size());
        if (e == cudaSuccess)
            e = cudaMemcpyAsync(d_loff, loff.data(), sizeof(long long) * loff.size(), cudaMemcpyHostToDevice, S->s0);
    }
    long long phase_off = 0;
    for (size_t w = 0; w < S->wfs.size() && e == cudaSuccess; ++w) {
        const WfsHost& W = S->wfs[w];
        if (W.n_valid > 0) {
            SensLaunch L{};
            L.ctx = make_ctx(S);
            L.real = S->cur;
            L.subaps = W.d_subaps;
            L.n_subaps = W.n_valid;
            L.sens = sens;
            L.P = P;
            e = launch_sens(L, W.p.n_fft, S->s0);
            ProjLaunch J{};
            J.ctx = L.ctx;
            J.real = S->cur;
            J.n_layers = S->n_layers;
            J.n_dms = S->n_dms;
            J.desc = S->d_dm_desc;
            J.g = S->d_dm_g;
            J.band = S->d_dm_band;
            J.act_map = S->d_dm_map;
            J.subaps = W.d_subaps;
            J.n_valid = W.n_valid;
            J.sens = sens;
            J.P = P;
            J.D = D;
            J.ld = ld;
            J.gvec = gvec;
            J.n_vec = n_vec;
            J.n_slopes = S->n_slopes;
            J.gc = gc;
            J.n_cmd = S->n_cmd;
            J.err = d_err;
            if (e == cudaSuccess && (D || gc)) e = launch_dm_adjoint(J, S->s0);
            if (e == cudaSuccess && (g_phase || g_layers))
                e = launch_phase_adjoint(J, g_phase, phase_total, phase_off, g_layers, loff[S->n_layers], d_loff, S->s0);
        }
        phase_off += (long long)W.N * W.N;
    }
    int h_err = 0;
    if (e == cudaSuccess) e = cudaStreamSynchronize(S->s0);
    if (e == cudaSuccess) e = cudaMemcpy(&h_err, d_err, sizeof(int), cudaMemcpyDeviceToHost);
    cudaFree(sens);
    cudaFree(d_err);
    cudaFree(d_loff);
    CK(e);
    if (h_err) return fail(S, MCAO_E_UNSUPPORTED, "a subaperture footprint meets more than 128 actuators per axis");
    return MCAO_OK;
}

// ------------------------------------------------------------------------------------------
// launch-shape tuning
// ------------------------------------------------------------------------------------------
static const int kTuneMin[kTuningKnobs] = {1, 25, 0, 1, 1, 1};
static const int kTuneMax[kTuningKnobs] = {8, 400, 1, 64, 2, 16};

static void tuning_to(const Tuning& t, int* v) {
    v[0] = t.sense_blocks_per_sm;
    v[1] = t.recon_ctas_pct;
    v[2] = t.science_after_aux;
    v[3] = t.tc_chunk;
    v[4] = t.multi_blocks_per_sm;
    v[5] = t.steps_per_graph;
}

static Tuning tuning_from(const int* v) {
    Tuning t;
    t.sense_blocks_per_sm = v[0];
    t.recon_ctas_pct = v[1];
    t.science_after_aux = v[2];
    t.tc_chunk = v[3];
    t.multi_blocks_per_sm = v[4];
    t.steps_per_graph = v[5];
    return t;
}

mcao_status mcao_get_tuning(const mcao_sim* S, int* values, int n) {
    if (!S || !values || n < kTuningKnobs) return MCAO_E_INVALID_ARG;
    tuning_to(S->tune, values);
    return MCAO_OK;
}

mcao_status mcao_set_tuning(mcao_sim* S, const int* values, int n) {
    if (!S || !values) return MCAO_E_INVALID_ARG;
    if (n != kTuningKnobs) return fail(S, MCAO_E_SHAPE, "%d tuning values, expected %d", n, kTuningKnobs);
    for (int i = 0; i < kTuningKnobs; ++i)
        if (values[i] < kTuneMin[i] || values[i] > kTuneMax[i])
            return fail(S, MCAO_E_INVALID_ARG, "tuning value %d = %d outside [%d, %d]", i, values[i], kTuneMin[i],
                        kTuneMax[i]);
    CK(cudaSetDevice(S->device));
    { mcao_status r_ = sync_all(S); if (r_ != MCAO_OK) return r_; }
    S->tune = tuning_from(values);
    release_graph(S);
    return MCAO_OK;
}

mcao_status mcao_autotune(mcao_sim* S, int steps_per_trial, int* values, int n, char* report, size_t report_len) {
    if (!S) return MCAO_E_INVALID_ARG;
    if (steps_per_trial < 1 || steps_per_trial > 100000)
        return fail(S, MCAO_E_INVALID_ARG, "steps_per_trial must be in [1, 100000]");
    if (values && n < kTuningKnobs) return fail(S, MCAO_E_SHAPE, "values needs %d entries", kTuningKnobs);
    if (!S->atm_loaded || !S->dms_loaded || !S->recon_loaded)
        return fail(S, MCAO_E_STATE, "load the atmosphere, the DMs and the reconstructor before tuning");
    if (S->profiling) return fail(S, MCAO_E_UNSUPPORTED, "switch the stage profiler off before tuning");
    CK(cudaSetDevice(S->device));
    // the trials advance the simulation: keep its state and restore it afterwards
    size_t sz = 0;
    mcao_status r = mcao_query(S, MCAO_Q_STATE, 0, &sz);
    if (r != MCAO_OK) return r;
    std::vector<char> blob(sz);
    if ((r = mcao_get_state(S, blob.data(), sz)) != MCAO_OK) return r;
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    CK(cudaEventCreate(&e0));
    CK(cudaEventCreate(&e1));
    auto trial = [&](float& ms) -> mcao_status {
        release_graph(S);
        mcao_status q = mcao_step(S, 2);   // builds the graph, warms up
        if (q != MCAO_OK) return q;
        CK(cudaEventRecord(e0, S->s0));
        if ((q = mcao_step(S, steps_per_trial)) != MCAO_OK) return q;
        CK(cudaEventRecord(e1, S->s0));
        CK(cudaEventSynchronize(e1));
        CK(cudaEventElapsedTime(&ms, e0, e1));
        ms /= (float)steps_per_trial;
        return sync_all(S);
    };
    // knobs that shape this configuration's step, with their candidates (the current value first)
    bool acf = false, fft = false;
    for (const auto& W : S->wfs) {
        if (W.n_valid == 0) continue;
        (W.fft_route ? fft : acf) = true;
    }
    const bool batched = S->n_real > 1;
    std::vector<std::pair<int, std::vector<int>>> knobs;
    if (acf) knobs.push_back({0, {2, 3, 4, 6}});
    if (!batched) knobs.push_back({1, {50, 75, 80, 85, 90, 95, 100, 125}});
    if (!S->sci.empty() && fft) knobs.push_back({2, {0, 1}});
    if (batched && S->tc) knobs.push_back({3, {4, 8, 16}});
    if (batched && !S->tc) knobs.push_back({4, {1, 2}});
    knobs.push_back({5, {1, 2, 4, 8}});
    int cur[kTuningKnobs];
    tuning_to(S->tune, cur);
    const char* names[kTuningKnobs] = {"sense_blocks_per_sm", "recon_ctas_pct", "science_after_aux", "tc_chunk",
                                       "multi_blocks_per_sm", "steps_per_graph"};
    std::string rep;
    float best_ms = 0.0f;
    r = trial(best_ms);
    char line[256];
    snprintf(line, sizeof(line), "start %.4f ms/step", best_ms);
    rep += line;
    for (auto& kn : knobs) {
        const int k = kn.first;
        int best = cur[k];
        rep += std::string("; ") + names[k] + ":";
        for (int c : kn.second) {
            if (r != MCAO_OK) break;
            int v[kTuningKnobs];
            std::copy(cur, cur + kTuningKnobs, v);
            v[k] = c;
            S->tune = tuning_from(v);
            float ms = 0.0f;
            r = trial(ms);
            snprintf(line, sizeof(line), " %d=%.4f", c, ms);
            rep += line;
            if (r == MCAO_OK && ms < best_ms) {
                best_ms = ms;
                best = c;
            }
        }
        cur[k] = best;
        snprintf(line, sizeof(line), " -> %d", best);
        rep += line;
    }
    S->tune = tuning_from(cur);
    release_graph(S);
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    mcao_status rs = mcao_set_state(S, blob.data(), sz);
    if (r != MCAO_OK) return r;
    if (rs != MCAO_OK) return rs;
    snprintf(line, sizeof(line), "; chosen %.4f ms/step", best_ms);
    rep += line;
    if (values) tuning_to(S->tune, values);
    if (report && report_len) {
        strncpy(report, rep.c_str(), report_len - 1);
        report[report_len - 1] = '\0';
    }
    return MCAO_OK;
}

mcao_status mcao_misreg_normal_equations(mcao_sim* S, int dm, const float* D_meas, size_t ld, double* JtJ, double* Jte,
                                         double* cost, double* meas_sq) {
    if (!S || !D_meas) return MCAO_E_INVALID_ARG;
    if (!S->atm_loaded || !S->dms_loaded) return fail(S, MCAO_E_STATE, "atmosphere and DMs must be loaded");
    if (dm < 0 || dm >= S->n_dms) return fail(S, MCAO_E_INVALID_ARG, "bad DM index");
    const int cmd0 = S->dm_cmd0[dm], n_cols = S->dm_cmd0[dm + 1] - cmd0;
    if (ld < (size_t)n_cols) return fail(S, MCAO_E_SHAPE, "ld must be >= %d (the DM's commands)", n_cols);
    CK(cudaSetDevice(S->device));
    int P = 1;
    for (const auto& W : S->wfs) P = std::max(P, W.p.n_px * W.p.n_px);
    CK(cudaDeviceSynchronize());   // D_meas may come from any stream
    { mcao_status r_ = sync_all(S); if (r_ != MCAO_OK) return r_; }
    float* sens = nullptr;
    double* rec = nullptr;
    cudaError_t e = dalloc(&sens, (size_t)S->n_slopes * P);
    if (e == cudaSuccess) e = cudaMalloc(&rec, sizeof(double) * ((size_t)S->n_slopes * 16 + 16));
    if (e == cudaSuccess) e = cudaMemsetAsync(rec, 0, sizeof(double) * (size_t)S->n_slopes * 16, S->s0);
    if (e == cudaSuccess) e = launch_dm_surfaces(make_dm_launch(S), S->s0);
    for (size_t w = 0; w < S->wfs.size() && e == cudaSuccess; ++w) {
        const WfsHost& W = S->wfs[w];
        if (W.n_valid == 0) continue;
        SensLaunch L{};
        L.ctx = make_ctx(S);
        L.real = S->cur;
        L.subaps = W.d_subaps;
        L.n_subaps = W.n_valid;
        L.sens = sens;
        L.P = P;
        e = launch_sens(L, W.p.n_fft, S->s0);
        ProjLaunch J{};
        J.ctx = L.ctx;
        J.real = S->cur;
        J.n_layers = S->n_layers;
        J.n_dms = S->n_dms;
        J.desc = S->d_dm_desc;
        J.g = S->d_dm_g;
        J.band = S->d_dm_band;
        J.act_map = S->d_dm_map;
        J.subaps = W.d_subaps;
        J.n_valid = W.n_valid;
        J.sens = sens;
        J.P = P;
        J.n_slopes = S->n_slopes;
        J.n_cmd = S->n_cmd;
        if (e == cudaSuccess) e = launch_misreg_gn(J, dm, D_meas, (long long)ld, cmd0, rec, S->s0);
    }
    double* out = rec + (size_t)S->n_slopes * 16;
    double h[16] = {0};
    if (e == cudaSuccess) e = launch_misreg_sum(rec, S->n_slopes, out, S->s0);
    if (e == cudaSuccess) e = cudaStreamSynchronize(S->s0);
    if (e == cudaSuccess) e = cudaMemcpy(h, out, sizeof(h), cudaMemcpyDeviceToHost);
    cudaFree(sens);
    cudaFree(rec);
    CK(e);
    // records: cost, Jte[4], upper triangle of JtJ row by row, sum D_meas^2
    if (cost) *cost = h[0];
    if (Jte)
        for (int p = 0; p < 4; ++p) Jte[p] = h[1 + p];
    if (JtJ) {
        int t = 5;
        for (int p = 0; p < 4; ++p)
            for (int q = p; q < 4; ++q, ++t) JtJ[p * 4 + q] = JtJ[q * 4 + p] = h[t];
    }
    if (meas_sq) *meas_sq = h[15];
    return MCAO_OK;
}

mcao_status mcao_interaction_matrix(mcao_sim* S, float* D, size_t ld) {
    if (!S || !D) return MCAO_E_INVALID_ARG;
    if (!S->atm_loaded || !S->dms_loaded) return fail(S, MCAO_E_STATE, "atmosphere and DMs must be loaded");
    if (ld < (size_t)S->n_cmd) return fail(S, MCAO_E_SHAPE, "ld must be >= %d", S->n_cmd);
    CK(cudaSetDevice(S->device));
    return run_adjoint(S, D, (long long)ld, nullptr, 0, nullptr, nullptr, nullptr);
}

mcao_status mcao_slopes_vjp(mcao_sim* S, const float* g_slopes, int n_vec, float* g_commands, float* g_phase,
                            float* g_layers) {
    if (!S || !g_slopes || n_vec < 1 || (!g_commands && !g_phase && !g_layers)) return MCAO_E_INVALID_ARG;
    if (!S->atm_loaded || !S->dms_loaded) return fail(S, MCAO_E_STATE, "atmosphere and DMs must be loaded");
    CK(cudaSetDevice(S->device));
    return run_adjoint(S, nullptr, 0, g_slopes, n_vec, g_commands, g_phase, g_layers);
}

mcao_status mcao_get_dm_surface(mcao_sim* S, int dm, float* out, size_t n) {
    if (!S || !out) return MCAO_E_INVALID_ARG;
    if (!S->dms_loaded) return fail(S, MCAO_E_STATE, "DMs not loaded");
    if (dm < 0 || dm >= S->n_dms) return fail(S, MCAO_E_INVALID_ARG, "bad DM index");
    size_t cnt = (size_t)S->dms[dm].surf_n * S->dms[dm].surf_n;
    if (n < cnt) return fail(S, MCAO_E_SHAPE, "need %zu samples", cnt);
    CK(cudaSetDevice(S->device));
    { mcao_status r_ = sync_all(S); if (r_ != MCAO_OK) return r_; }
    CK(launch_dm_surfaces(make_dm_launch(S), S->s0));
    CK(cudaStreamSynchronize(S->s0));
    CK(cudaMemcpy(out, S->d_dm_surf + (size_t)S->cur * S->surf_total + S->dm_desc[dm].surf_off, sizeof(float) * cnt,
                  cudaMemcpyDeviceToHost));
    return MCAO_OK;
}

mcao_status mcao_get_frames(mcao_sim* S, int wfs, float* lambda, int32_t* frames, size_t n) {
    if (!S) return MCAO_E_INVALID_ARG;
    if (!S->cfg.keep_frames) return fail(S, MCAO_E_STATE, "create the simulation with keep_frames = 1");
    if (wfs < 0 || wfs >= (int)S->wfs.size()) return fail(S, MCAO_E_INVALID_ARG, "bad WFS index");
    const WfsHost& W = S->wfs[wfs];
    size_t cnt = (size_t)W.n_valid * W.n_det * W.n_det;
    if (n < cnt) return fail(S, MCAO_E_SHAPE, "need %zu pixels", cnt);
    mcao_status r = MCAO_OK;
    const size_t off = (size_t)S->cur * S->n_frame_px + W.frame0;
    if (lambda) r = d2h(S, lambda, S->d_lam + off, sizeof(float) * cnt);
    if (r == MCAO_OK && frames) r = d2h(S, frames, S->d_frames + off, sizeof(int32_t) * cnt);
    return r;
}

mcao_status mcao_get_psf(mcao_sim* S, int sci, double* out, size_t n, double* sr_long, double* sr_last) {
    if (!S) return MCAO_E_INVALID_ARG;
    if (sci < 0 || sci >= (int)S->sci.size()) return fail(S, MCAO_E_INVALID_ARG, "bad science index");
    const Science& C = S->sci[sci];
    const size_t M = (size_t)C.M;
    if (out && n < M * M) return fail(S, MCAO_E_SHAPE, "need %zu pixels", M * M);
    SciAcc acc;
    mcao_status r = d2h(S, &acc, S->d_acc + (size_t)S->cur * S->sci.size() + sci, sizeof(acc));
    if (r != MCAO_OK) return r;
    if (sr_long) *sr_long = acc.n_sr ? acc.sr_sum / (double)acc.n_sr : 0.0;
    if (sr_last) *sr_last = acc.sr_last;
    if (out) {
        std::vector<double> t(M * M);
        r = d2h(S, t.data(), C.d_psf_t + (size_t)S->cur * M * M, sizeof(double) * M * M);
        if (r != MCAO_OK) return r;
        double norm = acc.n_psf ? 1.0 / ((double)acc.n_psf * C.sum_amp * C.sum_amp) : 0.0;
        for (size_t j = 0; j < M; ++j)
            for (size_t i = 0; i < M; ++i)
                out[j * M + i] = t[((i + M / 2) % M) * M + (j + M / 2) % M] * norm;
    }
    return MCAO_OK;
}

mcao_status mcao_check_bounded_wait(mcao_sim* S) {
    if (!S) return MCAO_E_INVALID_ARG;
    CK(cudaSetDevice(S->device));
    { mcao_status r_ = sync_all(S); if (r_ != MCAO_OK) return r_; }
    CK(launch_wait_probe(S->d_err, S->s0));
    return sync_all(S);   // reports the expired wait as MCAO_E_TIMEOUT and clears the flag
}

constexpr int kReadRing = 64;   // readout slots in flight at most

mcao_status mcao_read_async(mcao_sim* S, float* commands, double* strehl) {
    if (!S || (!commands && !strehl)) return MCAO_E_INVALID_ARG;
    if (commands && !S->dms_loaded) return fail(S, MCAO_E_STATE, "DMs not loaded");
    CK(cudaSetDevice(S->device));
    const int n_cmd = S->dms_loaded ? S->n_cmd : 0, n_sci = (int)S->sci.size();
    if (S->ring_ncmd != n_cmd || S->ring_nsci != n_sci) {
        // (re)size the ring after every earlier read has completed
        if (S->s_read) CK(cudaStreamSynchronize(S->s_read));
        dfree(S->d_ring_c);
        dfree(S->d_ring_s);
        CK(dalloc(&S->d_ring_c, (size_t)kReadRing * std::max(n_cmd, 1)));
        CK(dalloc(&S->d_ring_s, (size_t)kReadRing * 2 * std::max(n_sci, 1)));
        while ((int)S->ring_ready.size() < kReadRing) {
            cudaEvent_t a = nullptr, b = nullptr;
            CK(cudaEventCreateWithFlags(&a, cudaEventDisableTiming));
            CK(cudaEventCreateWithFlags(&b, cudaEventDisableTiming));
            S->ring_ready.push_back(a);
            S->ring_free.push_back(b);
        }
        S->ring_busy.assign(kReadRing, 0);
        S->ring_ncmd = n_cmd;
        S->ring_nsci = n_sci;
        S->ring_pos = 0;
    }
    mcao_status r = order_after_user(S);
    if (r != MCAO_OK) return r;
    const int slot = S->ring_pos;
    S->ring_pos = (S->ring_pos + 1) % kReadRing;
    float* rc = S->d_ring_c + (size_t)slot * std::max(n_cmd, 1);
    double* rs = S->d_ring_s + (size_t)slot * 2 * std::max(n_sci, 1);
    // the slot's previous copy to the host is done before the snapshot overwrites it
    if (S->ring_busy[slot]) CK(cudaStreamWaitEvent(S->s0, S->ring_free[slot], 0));
    const int nc = (commands && n_cmd > 0) ? n_cmd : 0, ns = strehl ? n_sci : 0;
    CK(launch_readout(S->d_c + (size_t)S->cur * std::max(n_cmd, 1), nc, S->d_acc + (size_t)S->cur * std::max(n_sci, 1),
                      ns, rc, rs, S->s0));
    CK(cudaEventRecord(S->ring_ready[slot], S->s0));
    CK(cudaStreamWaitEvent(S->s_read, S->ring_ready[slot], 0));
    if (nc) CK(cudaMemcpyAsync(commands, rc, sizeof(float) * nc, cudaMemcpyDeviceToHost, S->s_read));
    if (ns) CK(cudaMemcpyAsync(strehl, rs, sizeof(double) * 2 * ns, cudaMemcpyDeviceToHost, S->s_read));
    CK(cudaEventRecord(S->ring_free[slot], S->s_read));
    S->ring_busy[slot] = 1;
    r = signal_user(S);
    if (r != MCAO_OK) return r;
    // work queued on the caller's stream afterwards also sees the host copies
    if (S->user_set) CK(cudaStreamWaitEvent(S->user, S->ring_free[slot], 0));
    return MCAO_OK;
}

mcao_status mcao_get_marechal(mcao_sim* S, int sci, double* sr_long, double* sr_last) {
    if (!S) return MCAO_E_INVALID_ARG;
    if (sci < 0 || sci >= (int)S->sci.size()) return fail(S, MCAO_E_INVALID_ARG, "bad science index");
    SciAcc acc;
    mcao_status r = d2h(S, &acc, S->d_acc + (size_t)S->cur * S->sci.size() + sci, sizeof(acc));
    if (r != MCAO_OK) return r;
    if (sr_long) *sr_long = acc.n_sr ? std::exp(-acc.var_sum / (double)acc.n_sr) : 0.0;
    if (sr_last) *sr_last = std::exp(-acc.var_last);
    return MCAO_OK;
}

mcao_status mcao_reset_psf(mcao_sim* S) {
    if (!S) return MCAO_E_INVALID_ARG;
    CK(cudaSetDevice(S->device));
    { mcao_status r_ = sync_all(S); if (r_ != MCAO_OK) return r_; }
    const size_t NR = (size_t)S->n_real;
    for (auto& c : S->sci) CK(cudaMemsetAsync(c.d_psf_t, 0, sizeof(double) * NR * c.M * c.M, S->s0));
    CK(cudaMemsetAsync(S->d_acc, 0, sizeof(SciAcc) * NR * std::max<size_t>(S->sci.size(), 1), S->s0));
    CK(cudaStreamSynchronize(S->s0));
    return MCAO_OK;
}

mcao_status mcao_get_state(mcao_sim* S, void* buf, size_t n) {
    if (!S || !buf) return MCAO_E_INVALID_ARG;
    if (!S->dms_loaded) return fail(S, MCAO_E_STATE, "DMs not loaded");
    size_t need = 0;
    mcao_status r = mcao_query(S, MCAO_Q_STATE, 0, &need);
    if (r != MCAO_OK) return r;
    if (n < need) return fail(S, MCAO_E_SHAPE, "need %zu bytes", need);
    char* p = (char*)buf;
    StepState st;
    r = d2h(S, &st, S->d_st, sizeof(st));
    if (r != MCAO_OK) return r;
    int64_t hdr[4] = {0x4d43414f53544154LL, (int64_t)st.k_next, S->n_cmd, S->n_slopes};
    memcpy(p, hdr, sizeof(hdr));
    p += sizeof(hdr);
    for (int re = 0; re < S->n_real; ++re) {
        for (const float* src : {S->d_c, S->d_c_prev, S->d_dc_prev}) {
            if ((r = d2h(S, p, src + (size_t)re * S->n_cmd, sizeof(float) * S->n_cmd)) != MCAO_OK) return r;
            p += sizeof(float) * S->n_cmd;
        }
        if ((r = d2h(S, p, S->d_slopes + (size_t)re * S->n_slopes, sizeof(float) * S->n_slopes)) != MCAO_OK) return r;
        p += sizeof(float) * S->n_slopes;
        for (size_t q = 0; q < S->sci.size(); ++q) {
            if ((r = d2h(S, p, S->d_acc + (size_t)re * S->sci.size() + q, sizeof(SciAcc))) != MCAO_OK) return r;
            p += sizeof(SciAcc);
            const size_t mm = (size_t)S->sci[q].M * S->sci[q].M;
            if ((r = d2h(S, p, S->sci[q].d_psf_t + (size_t)re * mm, sizeof(double) * mm)) != MCAO_OK) return r;
            p += sizeof(double) * mm;
        }
    }
    return MCAO_OK;
}

mcao_status mcao_set_state(mcao_sim* S, const void* buf, size_t n) {
    if (!S || !buf) return MCAO_E_INVALID_ARG;
    if (!S->dms_loaded) return fail(S, MCAO_E_STATE, "DMs not loaded");
    size_t need = 0;
    mcao_status r = mcao_query(S, MCAO_Q_STATE, 0, &need);
    if (r != MCAO_OK) return r;
    if (n != need) return fail(S, MCAO_E_SHAPE, "checkpoint has %zu bytes, expected %zu", n, need);
    const char* p = (const char*)buf;
    int64_t hdr[4];
    memcpy(hdr, p, sizeof(hdr));
    if (hdr[0] != 0x4d43414f53544154LL || hdr[2] != S->n_cmd || hdr[3] != S->n_slopes || hdr[1] < 0)
        return fail(S, MCAO_E_SHAPE, "checkpoint does not match this configuration");
    p += sizeof(hdr);
    CK(cudaSetDevice(S->device));
    { mcao_status r_ = sync_all(S); if (r_ != MCAO_OK) return r_; }
    StepState st;
    st.k = hdr[1];
    st.k_next = hdr[1];
    CK(cudaMemcpyAsync(S->d_st, &st, sizeof(st), cudaMemcpyHostToDevice, S->s0));
    for (int re = 0; re < S->n_real; ++re) {
        for (float* dst : {S->d_c, S->d_c_prev, S->d_dc_prev}) {
            CK(cudaMemcpyAsync(dst + (size_t)re * S->n_cmd, p, sizeof(float) * S->n_cmd, cudaMemcpyHostToDevice, S->s0));
            p += sizeof(float) * S->n_cmd;
        }
        CK(cudaMemcpyAsync(S->d_slopes + (size_t)re * S->n_slopes, p, sizeof(float) * S->n_slopes,
                           cudaMemcpyHostToDevice, S->s0));
        p += sizeof(float) * S->n_slopes;
        for (size_t q = 0; q < S->sci.size(); ++q) {
            CK(cudaMemcpyAsync(S->d_acc + (size_t)re * S->sci.size() + q, p, sizeof(SciAcc), cudaMemcpyHostToDevice,
                               S->s0));
            p += sizeof(SciAcc);
            const size_t mm = (size_t)S->sci[q].M * S->sci[q].M;
            CK(cudaMemcpyAsync(S->sci[q].d_psf_t + (size_t)re * mm, p, sizeof(double) * mm, cudaMemcpyHostToDevice,
                               S->s0));
            p += sizeof(double) * mm;
        }
    }
    CK(cudaStreamSynchronize(S->s0));
    return MCAO_OK;
}

mcao_status mcao_set_sodium(mcao_sim* S, int wfs, double height, double na_fwhm) {
    if (!S) return MCAO_E_INVALID_ARG;
    if (wfs < 0 || wfs >= (int)S->wfs.size()) return fail(S, MCAO_E_INVALID_ARG, "bad WFS index");
    WfsHost& H = S->wfs[wfs];
    if (H.p.type != MCAO_WFS_LGS) return fail(S, MCAO_E_INVALID_ARG, "WFS %d is not a laser star", wfs);
    if (!(is_fin(height) && height > 0.0) || !(is_fin(na_fwhm) && na_fwhm >= 0.0))
        return fail(S, MCAO_E_INVALID_ARG, "height > 0 and na_fwhm >= 0 required");
    for (const auto& L : S->layers)
        if (L.alt_m >= height) return fail(S, MCAO_E_INVALID_ARG, "the laser star must stay above every layer");
    if (!wfs_variant_supported(H.p.n_px, H.p.n_fft, H.p.n_bin, na_fwhm > 0.0))
        return fail(S, MCAO_E_UNSUPPORTED, "WFS %d has no kernel for an elongated spot", wfs);
    CK(cudaSetDevice(S->device));
    { mcao_status r_ = sync_all(S); if (r_ != MCAO_OK) return r_; }
    H.p.height = height;
    H.p.na_fwhm = na_fwhm;
    for (auto& d : H.subaps) set_elongation(H, d);
    if (!H.subaps.empty())
        CK(cudaMemcpyAsync(H.d_subaps, H.subaps.data(), sizeof(SubapDev) * H.subaps.size(), cudaMemcpyHostToDevice,
                           S->s0));
    // block-per-subaperture sensors read their group's concatenated copy
    for (auto& g : S->fft_groups) {
        size_t off = 0;
        for (int w : g.wfs) {
            if (w == wfs && !H.subaps.empty())
                CK(cudaMemcpyAsync(g.d_subaps + off, H.subaps.data(), sizeof(SubapDev) * H.subaps.size(),
                                   cudaMemcpyHostToDevice, S->s0));
            off += S->wfs[w].subaps.size();
        }
    }
    return rebuild_views(S);   // cone projection of the new height (synchronises s0)
}

mcao_status mcao_set_controller(mcao_sim* S, double a1, double a2, double b0, double b1) {
    if (!S) return MCAO_E_INVALID_ARG;
    if (!is_fin(a1) || !is_fin(a2) || !is_fin(b0) || !is_fin(b1))
        return fail(S, MCAO_E_INVALID_ARG, "controller coefficients must be finite");
    if (!S->dms_loaded) return fail(S, MCAO_E_STATE, "load the DMs before setting the controller");
    CK(cudaSetDevice(S->device));
    { mcao_status r_ = sync_all(S); if (r_ != MCAO_OK) return r_; }
    S->use_ctl = true;
    S->ctl[0] = (float)a1; S->ctl[1] = (float)a2; S->ctl[2] = (float)b0; S->ctl[3] = (float)b1;
    const size_t n = (size_t)S->n_real * S->n_cmd;
    if (n) {
        CK(cudaMemcpyAsync(S->d_c_prev, S->d_c, sizeof(float) * n, cudaMemcpyDeviceToDevice, S->s0));
        CK(cudaMemsetAsync(S->d_dc_prev, 0, sizeof(float) * n, S->s0));
    }
    CK(cudaStreamSynchronize(S->s0));
    release_graph(S);
    return MCAO_OK;
}

mcao_status mcao_set_realization(mcao_sim* S, int r) {
    if (!S) return MCAO_E_INVALID_ARG;
    if (r < 0 || r >= S->n_real) return fail(S, MCAO_E_INVALID_ARG, "realization %d not in [0, %d)", r, S->n_real);
    S->cur = r;
    return MCAO_OK;
}

mcao_status mcao_set_profiling(mcao_sim* S, int on) {
    return mcao_set_profiling_stages(S, on ? (1u << MCAO_N_STAGES) - 1u : 0u);
}

mcao_status mcao_set_profiling_stages(mcao_sim* S, unsigned int mask) {
    if (!S) return MCAO_E_INVALID_ARG;
    if (mask >> MCAO_N_STAGES) return fail(S, MCAO_E_INVALID_ARG, "stage mask 0x%x has bits above the %d stages", mask,
                                           MCAO_N_STAGES);
    S->prof_mask = mask;
    S->profiling = mask != 0;
    S->prof_used = 0;
    S->prof_records.clear();
    S->prof_step_begin.clear();
    return MCAO_OK;
}

mcao_status mcao_get_profile(mcao_sim* S, double* ms, int64_t* counts, int n_stages, int64_t* launches_per_step) {
    if (!S) return MCAO_E_INVALID_ARG;
    CK(cudaSetDevice(S->device));
    { mcao_status r_ = sync_all(S); if (r_ != MCAO_OK) return r_; }
    std::vector<double> tot(ST_COUNT, 0.0);
    std::vector<int64_t> cnt(ST_COUNT, 0);
    for (auto& rec : S->prof_records) {
        float t = 0.0f;
        CK(cudaEventElapsedTime(&t, rec.second.first, rec.second.second));
        tot[rec.first] += t;
        cnt[rec.first] += 1;
    }
    for (int i = 0; i < n_stages && i < ST_COUNT; ++i) {
        if (ms) ms[i] = tot[i];
        if (counts) counts[i] = cnt[i];
    }
    if (launches_per_step) *launches_per_step = S->launches_per_step;
    S->prof_used = 0;
    S->prof_records.clear();
    S->prof_step_begin.clear();
    return MCAO_OK;
}

mcao_status mcao_get_timeline(mcao_sim* S, int32_t* stage, double* start_ms, double* end_ms, int32_t* step,
                              size_t n, size_t* n_total) {
    if (!S) return MCAO_E_INVALID_ARG;
    CK(cudaSetDevice(S->device));
    { mcao_status r_ = sync_all(S); if (r_ != MCAO_OK) return r_; }
    if (n_total) *n_total = S->prof_records.size();
    size_t out = 0;
    for (size_t q = 0; q < S->prof_step_begin.size(); ++q) {
        const size_t b = S->prof_step_begin[q];
        const size_t e = q + 1 < S->prof_step_begin.size() ? S->prof_step_begin[q + 1] : S->prof_records.size();
        if (b >= e) continue;
        cudaEvent_t origin = S->prof_records[b].second.first;
        for (size_t r = b; r < e && out < n; ++r, ++out) {
            const auto& rec = S->prof_records[r];
            float t0 = 0.0f, t1 = 0.0f;
            CK(cudaEventElapsedTime(&t0, origin, rec.second.first));
            CK(cudaEventElapsedTime(&t1, origin, rec.second.second));
            if (stage) stage[out] = rec.first;
            if (start_ms) start_ms[out] = t0;
            if (end_ms) end_ms[out] = t1;
            if (step) step[out] = (int32_t)q;
        }
    }
    return MCAO_OK;
}

mcao_status mcao_quantize_rows(const float* R, int rows, int cols, int ld, int dtype, void* codes, float* scales,
                               void* stream, char* err, size_t err_len) {
    auto bad = [&](mcao_status st, const char* msg) {
        if (err && err_len) snprintf(err, err_len, "%s", msg);
        return st;
    };
    if (dtype != MCAO_DTYPE_BF16 && dtype != MCAO_DTYPE_FP8_E4M3)
        return bad(MCAO_E_UNSUPPORTED, "dtype must be MCAO_DTYPE_BF16 or MCAO_DTYPE_FP8_E4M3");
    if (rows < 0 || cols < 0 || ld < cols) return bad(MCAO_E_INVALID_ARG, "rows, cols >= 0 and ld >= cols required");
    if (rows == 0 || cols == 0) return MCAO_OK;
    if (!R || !codes || (dtype == MCAO_DTYPE_FP8_E4M3 && !scales)) return bad(MCAO_E_INVALID_ARG, "null pointer");
    const int epv = 16 / recon_esize(dtype);
    if (cols % epv != 0) return bad(MCAO_E_SHAPE, "cols must be a multiple of 8 (BF16) or 16 (FP8 E4M3)");
    if (reinterpret_cast<uintptr_t>(codes) % 16 != 0) return bad(MCAO_E_SHAPE, "codes must be 16-byte aligned");
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    cudaError_t e = cudaSuccess;
    if (dtype == MCAO_DTYPE_FP8_E4M3) e = launch_recon_scales(R, rows, cols, ld, scales, st);
    if (e == cudaSuccess) e = launch_quantize_rows(R, rows, cols, ld, dtype, codes, scales, st);
    if (e != cudaSuccess) return bad(MCAO_E_CUDA, cudaGetErrorString(e));
    return MCAO_OK;
}

mcao_status mcao_generate_screen(int n, double pixel_m, double r0_m, double L0_m, uint64_t seed, float* out,
                                 void* stream, char* err, size_t err_len) {
    auto bad = [&](mcao_status st, const char* msg) {
        if (err && err_len) snprintf(err, err_len, "%s", msg);
        return st;
    };
    if (!out) return bad(MCAO_E_INVALID_ARG, "out is NULL");
    if (!(is_fin(pixel_m) && pixel_m > 0) || !(is_fin(r0_m) && r0_m > 0) || !(is_fin(L0_m) && L0_m > 0))
        return bad(MCAO_E_INVALID_ARG, "pixel, r0 and L0 must be finite and > 0");
    if (n < 2 || n > 4096) return bad(MCAO_E_SHAPE, "n must be in [2, 4096]");
    const std::vector<int> rad = factor_fft(n);
    if (rad.empty() || rad.size() > 16) return bad(MCAO_E_SHAPE, "n must be a product of 2, 3 and 5");
    int dev = 0, smem = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&smem, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
    if (e != cudaSuccess) return bad(MCAO_E_CUDA, cudaGetErrorString(e));
    if (screen_fft_smem(n) > (size_t)smem) return bad(MCAO_E_UNSUPPORTED, "n too large for the in-shared-memory FFT");
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    float2 *b = nullptr, *w = nullptr;
    e = cudaMallocAsync((void**)&b, sizeof(float2) * (size_t)n * n, st);
    if (e == cudaSuccess) e = cudaMallocAsync((void**)&w, sizeof(float2) * n, st);
    if (e == cudaSuccess) e = launch_screen(n, pixel_m, r0_m, L0_m, seed, rad.data(), (int)rad.size(), b, w, out, st);
    for (float2* p : {b, w})
        if (p) cudaFreeAsync(p, st);
    if (e != cudaSuccess) return bad(MCAO_E_CUDA, cudaGetErrorString(e));
    return MCAO_OK;
}

}  // extern "C"
