// ctu_api.cu -- C ABI of libctu.so (declared in include/ctu.h).
//
// Host side of the CTU-MHD integrator: argument validation, patch-list
// binding (patches grouped by shape so that every kernel launch covers a
// group of identical patches with no idle blocks), scratch management, the
// CFL reduction of Eq. (Ca), the step launch sequence, flux-register
// binding, the sticky device status and the optional per-kernel timers.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <array>
#include <cstdint>
#include <cstdlib>
#include <cstring>
#include <map>
#include <new>
#include <string>
#include <vector>

#include "ctu.h"
#include "amr_ops.cuh"
#include "tag_ops.cuh"
#include "ctu_launch.h"

using namespace ctu;

// Per-kernel CUDA-event timing: an event is recorded on the launching stream
// right before and right after every kernel group; totals are resolved on read.
struct EventProf : ProfHook {
    struct Rec { const char *name; cudaEvent_t a, b; };
    std::vector<cudaEvent_t> pool;
    size_t used = 0;
    std::vector<Rec> pending;
    const char *open = nullptr;
    cudaEvent_t open_ev = nullptr;
    std::vector<std::string> names;
    std::map<std::string, std::pair<double, long long>> tot;
    cudaEvent_t take()
    {
        if (used == pool.size()) {
            cudaEvent_t e;
            if (cudaEventCreate(&e) != cudaSuccess) return nullptr;
            pool.push_back(e);
        }
        return pool[used++];
    }
    void mark(const char *name, cudaStream_t s) override
    {
        cudaEvent_t e = take();
        if (!e) return;
        cudaEventRecord(e, s);
        if (name) {
            open = name;
            open_ev = e;
        } else if (open) {
            pending.push_back({open, open_ev, e});
            open = nullptr;
        }
    }
    void resolve()
    {
        for (const Rec &r : pending) {
            float ms = 0.f;
            if (cudaEventElapsedTime(&ms, r.a, r.b) == cudaSuccess) {
                if (tot.find(r.name) == tot.end()) {
                    names.push_back(r.name);
                    tot[r.name] = {0.0, 0};
                }
                tot[r.name].first += ms;
                tot[r.name].second += 1;
            }
        }
        pending.clear();
        used = 0;
    }
    void reset()
    {
        pending.clear();
        used = 0;
        names.clear();
        tot.clear();
    }
    ~EventProf() override
    {
        for (cudaEvent_t e : pool) cudaEventDestroy(e);
    }
};

// Key of a patch shape in the autotune cache.
static std::array<int, 3> shape_key(const int *n) { return {n[0], n[1], n[2]}; }

// Every kernel's block count over a batch fits one launch (grid x < 2^31).
static bool grid_fits(const std::vector<Group> &gs, int ndim)
{
    long long tot[8] = {0, 0, 0, 0, 0, 0, 0, 0};
    for (const Group &G : gs) {
        const long long c = G.count;
        tot[0] += c * Tiles::ghosted(G.N);
        for (int D = 0; D < 3; ++D) {
            // (one row per thread: the most blocks the x kernels launch)
            tot[1 + D] += c * Tiles::div1(G.n, ndim, D, G.xw, G.seg, true, 1);
            tot[4 + D] += c * (D == 0 ? Tiles::sweep_x(G.n, G.xw, 1) : Tiles::sweep_m(G.n, D, G.xw, G.seg));
        }
        tot[7] += c * Tiles::interior(G.n, G.xw);
    }
    for (long long t : tot)
        if (t >= (1LL << 31)) return false;
    return true;
}

struct ctu_ctx {
    ctu_config cfg;
    // autotuned thread-tile width along x and marching segment per shape
    std::map<std::array<int, 3>, std::array<int, 2>> tune;
    bool tuning = false;  // steps of ctu_autotune leave the flux registers alone
    // device copies of the level-operator descriptors (prolong, restrict,
    // reflux, tiled and flat tagging, exchange copy / pack / unpack),
    // re-uploaded when a call brings different contents
    std::vector<char> opcache[8];
    void *optab[8] = {nullptr, nullptr, nullptr, nullptr, nullptr, nullptr, nullptr, nullptr};
    size_t opcap[8] = {0, 0, 0, 0, 0, 0, 0, 0};
    int device = 0;
    int sms = 152;  // streaming multiprocessors of the device
    // patch list cache (caller order) and its device table (grouped order)
    std::vector<ctu_patch> hpatch;
    std::vector<int> sorted_of;  // caller index -> device-table index
    std::vector<Group> groups;
    DevPatch *dpatch = nullptr;
    int dpatch_cap = 0;
    long long sstride = 0;
    double dxmin = 0.0;
    // scratch
    void *scratch = nullptr;
    size_t scratch_bytes = 0;
    // status, reduction word, per-step parameters
    unsigned int *dstatus = nullptr;
    unsigned long long *dmax = nullptr;
    unsigned long long *dfloor = nullptr;  // cells the floors changed
    unsigned long long *dtagcnt = nullptr;  // per-patch tag counts when the caller gives none
    int dtagcnt_cap = 0;
    StepParams *dsp = nullptr;
    // flux registers
    std::vector<ctu_flux_window> hwin;
    double *reg = nullptr;
    DevWindow *dwin = nullptr;
    int *dwstart = nullptr;  // npatch * 3 CSR bases, then the plane positions
    int dwin_cap = 0, dws_cap = 0;
    int dwin_n = 0;      // windows in dwin
    int dwin_faces = 0;  // most faces of one of them within its patch
    bool win_dirty = false;
    int last_launches = 0;
    EventProf *prof = nullptr;
};

static ctu_status cuda_fail(cudaError_t e)
{
    return e == cudaErrorMemoryAllocation ? CTU_ENOMEM : CTU_ECUDA;
}

#define CTU_CUDA(call)                               \
    do {                                             \
        cudaError_t e_ = (call);                     \
        if (e_ != cudaSuccess) return cuda_fail(e_); \
    } while (0)

static int active_ghost(const ctu_ctx *ctx, int d) { return d < ctx->cfg.ndim ? 4 : 0; }

static ctu_status validate_patches(const ctu_ctx *ctx, int64_t stride, const ctu_patch *p, int np)
{
    if (!p || np <= 0 || np > 65535) return CTU_EINVAL;
    for (int i = 0; i < np; ++i) {
        long long cells = 1;
        for (int d = 0; d < 3; ++d) {
            if (p[i].n[d] < 1 || p[i].n[d] > 4096) return CTU_EINVAL;
            if (d >= ctx->cfg.ndim && p[i].n[d] != 1) return CTU_EINVAL;
            if (!(p[i].dx[d] > 0.0)) return CTU_EINVAL;
            cells *= (long long)p[i].n[d] + 2 * active_ghost(ctx, d);
        }
        if (cells > (1LL << 30)) return CTU_EINVAL;  // local cell indices are 32-bit
        if (p[i].base < 0 || p[i].base + cells > stride) return CTU_EINVAL;
    }
    return CTU_OK;
}

// Device table of flux windows, sorted by (device patch index, dir, plane),
// with a per-(patch, dir) CSR index over planes (see StepArgs::wbase).
// Windows of patches beyond the bound list, or with a plane outside
// [0, n_dir], are ignored.
static ctu_status upload_windows(ctu_ctx *ctx, cudaStream_t s)
{
    const int np = (int)ctx->hpatch.size();
    ctx->dwin_n = 0;
    ctx->dwin_faces = 0;
    if (!ctx->reg || ctx->hwin.empty() || np == 0) {
        ctx->win_dirty = false;
        return CTU_OK;
    }
    struct W { long long key; int n_d; DevWindow w; };
    std::vector<W> v;
    int faces = 0;
    for (const ctu_flux_window &x : ctx->hwin) {
        if (x.patch >= np) continue;
        if (x.plane > ctx->hpatch[x.patch].n[x.dir]) continue;
        {  // faces of the window within the patch
            const int *pn = ctx->hpatch[x.patch].n;
            const int ea = x.dir == 0 ? 1 : 0, eb = x.dir == 2 ? 1 : 2;
            const long long fa = std::max(0, std::min(x.a1, pn[ea]) - x.a0);
            const long long fb = std::max(0, std::min(x.b1, pn[eb]) - x.b0);
            faces = (int)std::max<long long>(faces, std::min<long long>(fa * fb, 1ll << 30));
        }
        DevWindow w;
        w.patch = ctx->sorted_of[x.patch];
        w.dir = x.dir; w.plane = x.plane; w.a0 = x.a0; w.a1 = x.a1; w.b0 = x.b0; w.b1 = x.b1; w.pad = 0;
        w.weight = x.weight;
        w.dst = x.dst;
        v.push_back({((long long)(w.patch * 3 + w.dir) << 20) + w.plane, ctx->hpatch[x.patch].n[x.dir], w});
    }
    std::stable_sort(v.begin(), v.end(), [](const W &a, const W &b) { return a.key < b.key; });
    std::vector<DevWindow> dw(v.size() ? v.size() : 1);
    for (size_t i = 0; i < v.size(); ++i) dw[i] = v[i].w;
    // CSR: wbase (3 np entries) followed by the plane positions
    std::vector<int> sc(3 * np, -1);
    size_t i = 0;
    while (i < v.size()) {
        const int pd = (int)(v[i].key >> 20);
        const int n_d = v[i].n_d;
        const int base = (int)sc.size();
        sc[pd] = base - 3 * np;
        sc.resize(sc.size() + n_d + 2, 0);
        size_t j = i;
        for (int pl = 0; pl <= n_d + 1; ++pl) {
            while (j < v.size() && (int)(v[j].key >> 20) == pd && v[j].w.plane < pl) ++j;
            sc[base + pl] = (int)j;
        }
        while (i < v.size() && (int)(v[i].key >> 20) == pd) ++i;
    }
    if ((int)dw.size() > ctx->dwin_cap) {
        if (ctx->dwin) cudaFree(ctx->dwin);
        ctx->dwin = nullptr;
        CTU_CUDA(cudaMalloc(&ctx->dwin, sizeof(DevWindow) * dw.size()));
        ctx->dwin_cap = (int)dw.size();
    }
    if ((int)sc.size() > ctx->dws_cap) {
        if (ctx->dwstart) cudaFree(ctx->dwstart);
        ctx->dwstart = nullptr;
        CTU_CUDA(cudaMalloc(&ctx->dwstart, sizeof(int) * sc.size()));
        ctx->dws_cap = (int)sc.size();
    }
    CTU_CUDA(cudaMemcpyAsync(ctx->dwin, dw.data(), sizeof(DevWindow) * dw.size(), cudaMemcpyHostToDevice, s));
    CTU_CUDA(cudaMemcpyAsync(ctx->dwstart, sc.data(), sizeof(int) * sc.size(), cudaMemcpyHostToDevice, s));
    CTU_CUDA(cudaStreamSynchronize(s));
    ctx->dwin_n = (int)v.size();
    ctx->dwin_faces = faces;
    ctx->win_dirty = false;
    return CTU_OK;
}

// Upload the patch list (grouped by shape) if it differs from the cached one.
static ctu_status bind_patches(ctu_ctx *ctx, const ctu_patch *p, int np, cudaStream_t s)
{
    if ((int)ctx->hpatch.size() == np && std::memcmp(ctx->hpatch.data(), p, sizeof(ctu_patch) * np) == 0) {
        if (ctx->win_dirty) return upload_windows(ctx, s);
        return CTU_OK;
    }
    std::vector<int> order(np);
    for (int i = 0; i < np; ++i) order[i] = i;
    std::stable_sort(order.begin(), order.end(), [&](int a, int b) {
        for (int d = 0; d < 3; ++d)
            if (p[a].n[d] != p[b].n[d]) return p[a].n[d] < p[b].n[d];
        return false;
    });
    std::vector<DevPatch> dp(np);
    std::vector<int> sorted_of(np);
    std::vector<Group> groups;
    long long off = 0;
    double dxmin = 1e300;
    for (int r = 0; r < np; ++r) {
        const ctu_patch &src = p[order[r]];
        sorted_of[order[r]] = r;
        DevPatch &q = dp[r];
        long long cells = 1;
        q.hmin = 1e300;
        for (int d = 0; d < 3; ++d) {
            q.n[d] = src.n[d];
            q.g[d] = active_ghost(ctx, d);
            q.N[d] = q.n[d] + 2 * q.g[d];
            q.dx[d] = src.dx[d];
            q.idx[d] = 1.0 / src.dx[d];
            q.idxf[d] = (float)q.idx[d];
            cells *= q.N[d];
            if (d < ctx->cfg.ndim) {
                q.hmin = std::min(q.hmin, q.dx[d]);
                dxmin = std::min(dxmin, q.dx[d]);
            }
        }
        q.base = src.base;
        q.soff = off;
        off += (cells + 31) / 32 * 32;
        if (groups.empty() || std::memcmp(groups.back().n, q.n, sizeof(q.n)) != 0) {
            Group G;
            G.first = r;
            G.count = 0;
            for (int d = 0; d < 3; ++d) { G.n[d] = q.n[d]; G.N[d] = q.N[d]; }
            groups.push_back(G);
        }
        groups.back().count += 1;
    }
    // tile parameters per shape (autotuned, else the default rule), and the
    // launch order: largest patches first
    std::vector<Group> g2(groups.rbegin(), groups.rend());
    for (Group &G : g2) {
        const auto it = ctx->tune.find(shape_key(G.n));
        G.xw = it != ctx->tune.end() ? it->second[0] : Tiles::xw(G.n[0]);
        G.seg = it != ctx->tune.end() ? it->second[1] : SEG;
    }
    if (!grid_fits(g2, ctx->cfg.ndim)) return CTU_EINVAL;
    if (np > ctx->dpatch_cap) {
        if (ctx->dpatch) cudaFree(ctx->dpatch);
        ctx->dpatch = nullptr;
        CTU_CUDA(cudaMalloc(&ctx->dpatch, sizeof(DevPatch) * np));
        ctx->dpatch_cap = np;
    }
    CTU_CUDA(cudaMemcpyAsync(ctx->dpatch, dp.data(), sizeof(DevPatch) * np, cudaMemcpyHostToDevice, s));
    CTU_CUDA(cudaStreamSynchronize(s));
    ctx->hpatch.assign(p, p + np);
    ctx->sorted_of = sorted_of;
    ctx->groups = g2;
    ctx->sstride = off;
    ctx->dxmin = dxmin;
    return upload_windows(ctx, s);
}

// Scratch layout: SCRATCH_ARRAYS planes of the working precision, then (each
// 256-byte aligned) the shock flags of the hybrid integration (one byte per
// scratch cell) and, with the parabolic terms, L_P^n (seven words of the
// working precision), the half-step fields (one 8-byte plane, T; eight
// with viscosity, resistivity or anisotropic conduction) and the face fluxes
// of the parabolic face pass (3 directions x 7 words of the working
// precision) per scratch cell, and L_P^(n+1/2) (7 words of the working
// precision) differenced from them for the x sweep's update.
struct ScratchOffsets {
    size_t flags, lp, th, pif, lph, total;
};
static size_t align256(size_t b) { return (b + 255) / 256 * 256; }
static ScratchOffsets scratch_offsets(const ctu_ctx *ctx)
{
    const size_t elt = ctx->cfg.precision == CTU_FP64 ? sizeof(double) : sizeof(float);
    const size_t S = (size_t)ctx->sstride;
    ScratchOffsets o;
    o.flags = align256((size_t)SCRATCH_ARRAYS * S * elt);
    const double kpar = ctx->cfg.kappa_par > 0.0 ? ctx->cfg.kappa_par : ctx->cfg.kappa;
    const bool tensor = ctx->cfg.nu > 0.0 || ctx->cfg.eta > 0.0 || kpar != ctx->cfg.kappa || ctx->cfg.tc_phi > 0.0;
    const bool par = ctx->cfg.kappa > 0.0 || kpar > 0.0 || tensor;
    o.lp = align256(o.flags + (ctx->cfg.shock_detect ? S : 0));
    o.th = align256(o.lp + (par ? 7 * S * elt : 0));
    o.pif = align256(o.th + (par ? (tensor ? 8 : 1) * S * sizeof(double) : 0));
    o.lph = align256(o.pif + (par ? 3 * 7 * S * elt : 0));
    o.total = o.lph + (par ? 7 * S * elt : 0);
    return o;
}

static ctu_status ensure_scratch(ctu_ctx *ctx)
{
    const size_t need = scratch_offsets(ctx).total;
    if (need <= ctx->scratch_bytes) return CTU_OK;
    if (ctx->scratch) {
        CTU_CUDA(cudaDeviceSynchronize());
        cudaFree(ctx->scratch);
        ctx->scratch = nullptr;
        ctx->scratch_bytes = 0;
    }
    CTU_CUDA(cudaMalloc(&ctx->scratch, need));
    ctx->scratch_bytes = need;
    return CTU_OK;
}

static StepArgs make_args(const ctu_ctx *ctx, const double *Uin, double *Uout, int64_t stride, int np,
                          const double *dtch)
{
    StepArgs a;
    std::memset(&a, 0, sizeof(a));
    a.patches = ctx->dpatch;
    a.npatch = np;
    a.ndim = ctx->cfg.ndim;
    // the relativistic path reads gam == 0 as the Taub-Mathews equation of state
    const bool tm = ctx->cfg.eos == CTU_EOS_TM;
    a.gam = tm ? 0.0 : ctx->cfg.gamma;
    a.igm = tm ? 0.0 : 1.0 / (ctx->cfg.gamma - 1.0);
    a.gamf = (float)a.gam;
    a.gm1f = tm ? 0.0f : (float)(ctx->cfg.gamma - 1.0);
    a.glm_alpha = ctx->cfg.glm_alpha;
    a.upwind = ctx->cfg.trace_mode;
    a.limiter = ctx->cfg.recon;
    a.shock_eps = ctx->cfg.shock_eps;
    a.shock_q = ctx->cfg.shock_q;
    a.flags = nullptr;
    a.kappa = ctx->cfg.kappa;
    a.kpar = ctx->cfg.kappa_par > 0.0 ? ctx->cfg.kappa_par : ctx->cfg.kappa;
    a.nu = ctx->cfg.nu;
    a.eta = ctx->cfg.eta;
    a.kappaf = (float)ctx->cfg.kappa;
    a.dkappaf = (float)(a.kpar - a.kappa);
    a.kmaxf = (float)(a.kpar > a.kappa ? a.kpar : a.kappa);
    a.nuf = (float)ctx->cfg.nu;
    a.etaf = (float)ctx->cfg.eta;
    a.par_cond = a.kappa > 0.0 || a.kpar > 0.0;
    a.par_visc = ctx->cfg.nu > 0.0;
    a.par_res = ctx->cfg.eta > 0.0;
    a.par_aniso = a.kpar != a.kappa;
    a.phi = ctx->cfg.tc_phi;
    a.phif = (float)ctx->cfg.tc_phi;
    a.par_sat = a.par_cond && ctx->cfg.tc_phi > 0.0;
    a.gm1lo = tm ? 0.0f : (float)((ctx->cfg.gamma - 1.0) - (double)a.gm1f);
    a.lp = nullptr;
    a.th = nullptr;
    a.pif = nullptr;
    a.lph = nullptr;
    if (ctx->scratch) {
        const ScratchOffsets o = scratch_offsets(ctx);
        if (ctx->cfg.shock_detect) a.flags = (unsigned char *)ctx->scratch + o.flags;
        if (a.par_cond || a.par_visc || a.par_res) {
            a.lp = (const unsigned char *)ctx->scratch + o.lp;
            a.th = (double *)((unsigned char *)ctx->scratch + o.th);
            a.pif = (unsigned char *)ctx->scratch + o.pif;
            a.lph = (unsigned char *)ctx->scratch + o.lph;
        }
    }
    a.U = Uin;
    a.Uout = Uout;
    a.ustride = stride;
    a.sstride = ctx->sstride;
    a.dtch = dtch;
    a.sp = ctx->dsp;
    a.status = ctx->dstatus;
    const bool regs = ctx->reg && !ctx->hwin.empty() && !ctx->tuning;
    a.win = regs ? ctx->dwin : nullptr;
    a.nwin = regs ? ctx->dwin_n : 0;
    a.wfaces = regs ? ctx->dwin_faces : 0;
    a.wbase = regs ? ctx->dwstart : nullptr;
    a.wpos = regs ? ctx->dwstart + 3 * (int)ctx->hpatch.size() : nullptr;
    a.reg = regs ? ctx->reg : nullptr;
    a.nextmax = nullptr;
    return a;
}

static LaunchInfo make_info(const ctu_ctx *ctx)
{
    LaunchInfo li;
    li.groups = ctx->groups.data();
    li.ngroups = (int)ctx->groups.size();
    const int r = ctx->cfg.recon;
    const bool ref = ctx->cfg.trace_mode >= CTU_TRACE_CENTER;
    const bool hyb = ctx->cfg.shock_detect != 0;
    const bool hllc = ctx->cfg.physics == CTU_MHD && ctx->cfg.riemann == CTU_HLLC;
    const bool par = ctx->cfg.kappa > 0.0 || ctx->cfg.kappa_par > 0.0 || ctx->cfg.nu > 0.0 || ctx->cfg.eta > 0.0;
    li.recon = r == CTU_PPM
                   ? (par ? RECON_PPM_PAR
                          : (hllc ? RECON_PPM_HLLC : (hyb ? RECON_PPM_HYB : (ref ? RECON_PPM_REF : RECON_PPM))))
             : r == CTU_LINEAR_MC
                   ? (par ? RECON_MC_PAR
                          : (hllc ? RECON_MC_HLLC : (hyb ? RECON_MC_HYB : (ref ? RECON_MC_REF : RECON_MC))))
             : r == CTU_WENO3 ? RECON_WENO3 : RECON_LIN;
    if (ctx->cfg.corner == CTU_CORNER_MT) li.recon = r == CTU_PPM ? RECON_PPM_MT : RECON_MC_MT;
    li.iface64 = ctx->cfg.precision == CTU_MIXED_IFACE64;
    li.physics = ctx->cfg.physics == CTU_SRMHD ? PH_SR : PH_MHD;
    li.scratch = ctx->scratch;
    li.sp = ctx->dsp;
    li.prof = ctx->prof;
    li.sms = ctx->sms;
    return li;
}

namespace ctu {
template <> int launch_step<double>(const StepArgs &a, const LaunchInfo &li, cudaStream_t s)
{
    if (li.physics == PH_SR) return launch_step_sr<double>(a, li, s);
    if (recon_mt(li.recon)) return launch_step_mt<double, 1>(a, li, s);
    if (recon_par(li.recon)) return launch_step_var<double, 1, 4>(a, li, s);
    if (recon_hllc(li.recon)) return launch_step_var<double, 1, 3>(a, li, s);
    if (recon_hybrid(li.recon)) return launch_step_var<double, 1, 2>(a, li, s);
    if (li.recon >= RECON_PPM_REF) return launch_step_var<double, 1, 1>(a, li, s);
    return li.recon >= RECON_LIN ? launch_step_var<double, 1, 0>(a, li, s) : launch_step_impl<double, 1>(a, li, s);
}
template <> int launch_step<float>(const StepArgs &a, const LaunchInfo &li, cudaStream_t s)
{
    if (li.physics == PH_SR) return launch_step_sr<float>(a, li, s);
    if (recon_mt(li.recon)) return launch_step_mt<float, 0>(a, li, s);
    if (recon_par(li.recon)) return launch_step_var<float, 0, 4>(a, li, s);
    if (recon_hllc(li.recon)) return launch_step_var<float, 0, 3>(a, li, s);
    if (recon_hybrid(li.recon)) return launch_step_var<float, 0, 2>(a, li, s);
    if (li.recon >= RECON_PPM_REF) return launch_step_var<float, 0, 1>(a, li, s);
    if (li.recon >= RECON_LIN) return launch_step_var<float, 0, 0>(a, li, s);
    return li.iface64 ? launch_step_impl<float, 1>(a, li, s) : launch_step_impl<float, 0>(a, li, s);
}
} // namespace ctu

__global__ void k_dt_finalize(const unsigned long long *m, double cfl, double dxmin, double *dtch)
{
    const double M = __longlong_as_double((long long)*m);
    const double dt = cfl / M;
    dtch[0] = dt;
    dtch[1] = cfl * dxmin / dt;
}

extern "C" {

ctu_status ctu_init(const ctu_config *cfg, ctu_ctx **out)
{
    if (!cfg || !out) return CTU_EINVAL;
    *out = nullptr;
    if (cfg->physics != CTU_MHD && cfg->physics != CTU_SRMHD) return CTU_EINVAL;
    if (cfg->eos != CTU_EOS_IDEAL && cfg->eos != CTU_EOS_TM) return CTU_EINVAL;
    // the Taub-Mathews equation of state belongs to relativistic MHD
    if (cfg->eos == CTU_EOS_TM && cfg->physics != CTU_SRMHD) return CTU_EUNSUPPORTED;
    if (cfg->eos == CTU_EOS_IDEAL && !(cfg->gamma > 1.0)) return CTU_EINVAL;
    if (cfg->ndim < 1 || cfg->ndim > 3) return CTU_EINVAL;
    if (cfg->recon < CTU_LINEAR_MC || cfg->recon > CTU_WENO3) return CTU_EINVAL;
    if (cfg->predictor != CTU_CHAR_TRACE && cfg->predictor != CTU_MUSCL_HANCOCK) return CTU_EINVAL;
    if (cfg->riemann != CTU_HLLD && cfg->riemann != CTU_HLL && cfg->riemann != CTU_HLLC) return CTU_EINVAL;
    // implemented combinations: MHD with characteristic tracing + HLLD (or
    // HLLC with PPM / MC-linear, trace modes ALL / UPWIND, FP64 or CTU_MIXED,
    // no hybrid integration); SRMHD with MUSCL-Hancock (MC-linear primitive
    // slopes) + HLL
    if (cfg->physics == CTU_MHD && (cfg->predictor != CTU_CHAR_TRACE || cfg->riemann == CTU_HLL))
        return CTU_EUNSUPPORTED;
    if (cfg->physics == CTU_MHD && cfg->riemann == CTU_HLLC &&
        ((cfg->recon != CTU_PPM && cfg->recon != CTU_LINEAR_MC) || cfg->trace_mode > CTU_TRACE_UPWIND ||
         cfg->precision == CTU_MIXED_IFACE64 || cfg->shock_detect))
        return CTU_EUNSUPPORTED;
    if (cfg->physics == CTU_SRMHD &&
        (cfg->predictor != CTU_MUSCL_HANCOCK || cfg->riemann != CTU_HLL || cfg->recon != CTU_LINEAR_MC ||
         cfg->precision == CTU_MIXED_IFACE64))
        return CTU_EUNSUPPORTED;
    if (cfg->precision != CTU_FP64 && cfg->precision != CTU_MIXED && cfg->precision != CTU_MIXED_IFACE64)
        return CTU_EINVAL;
    // the other reconstructions are built for the FP64 and CTU_MIXED paths
    if ((cfg->recon > CTU_PPM || cfg->trace_mode > CTU_TRACE_UPWIND) && cfg->precision == CTU_MIXED_IFACE64)
        return CTU_EUNSUPPORTED;
    if (!(cfg->cfl > 0.0 && cfg->cfl <= 1.0)) return CTU_EINVAL;
    if (!(cfg->glm_alpha >= 0.0)) return CTU_EINVAL;
    if (cfg->nghost != 4) return CTU_EINVAL;
    if (cfg->trace_mode < CTU_TRACE_ALL || cfg->trace_mode > CTU_TRACE_CW84) return CTU_EINVAL;
    if (!(cfg->p_floor >= 0.0 && cfg->p_floor < INFINITY) || !(cfg->rho_floor >= 0.0 && cfg->rho_floor < INFINITY))
        return CTU_EINVAL;
    if (cfg->physics == CTU_SRMHD && (cfg->p_floor != 0.0 || cfg->rho_floor != 0.0)) return CTU_EUNSUPPORTED;
    if (cfg->shock_detect != 0 && cfg->shock_detect != 1) return CTU_EINVAL;
    if (cfg->shock_detect) {
        if (!(cfg->shock_eps > 0.0 && cfg->shock_eps < INFINITY) || (cfg->shock_q != 0 && cfg->shock_q != 1))
            return CTU_EINVAL;
        // the hybrid integration: ideal MHD, PPM or MC-linear, tracing
        // without or with the w_(+/-) reference, FP64 or CTU_MIXED
        if (cfg->physics != CTU_MHD || (cfg->recon != CTU_PPM && cfg->recon != CTU_LINEAR_MC) ||
            cfg->trace_mode > CTU_TRACE_UPWIND || cfg->precision == CTU_MIXED_IFACE64)
            return CTU_EUNSUPPORTED;
    }
    if (!(cfg->kappa >= 0.0 && cfg->kappa < INFINITY) || !(cfg->nu >= 0.0 && cfg->nu < INFINITY) ||
        !(cfg->eta >= 0.0 && cfg->eta < INFINITY) || !(cfg->kappa_par >= 0.0 && cfg->kappa_par < INFINITY) ||
        !(cfg->tc_phi >= 0.0 && cfg->tc_phi < INFINITY))
        return CTU_EINVAL;
    // the parabolic terms: ideal MHD, PPM or MC-linear, HLLD, tracing without
    // or with the w_(+/-) reference, no hybrid integration, FP64 or CTU_MIXED
    if ((cfg->kappa > 0.0 || cfg->kappa_par > 0.0 || cfg->nu > 0.0 || cfg->eta > 0.0) &&
        (cfg->physics != CTU_MHD || (cfg->recon != CTU_PPM && cfg->recon != CTU_LINEAR_MC) ||
         cfg->riemann != CTU_HLLD || cfg->trace_mode > CTU_TRACE_UPWIND || cfg->shock_detect ||
         cfg->precision == CTU_MIXED_IFACE64))
        return CTU_EUNSUPPORTED;
    if (cfg->corner != CTU_CORNER_CELL && cfg->corner != CTU_CORNER_MT) return CTU_EINVAL;
    // the corner coupling of Mignone & Tzeferacos: Pi = 0, ideal MHD, PPM or
    // MC-linear, HLLD, trace modes ALL / UPWIND, FP64 or CTU_MIXED
    if (cfg->corner == CTU_CORNER_MT &&
        (cfg->physics != CTU_MHD || (cfg->recon != CTU_PPM && cfg->recon != CTU_LINEAR_MC) ||
         cfg->riemann != CTU_HLLD || cfg->trace_mode > CTU_TRACE_UPWIND || cfg->shock_detect ||
         cfg->precision == CTU_MIXED_IFACE64 || cfg->kappa > 0.0 || cfg->kappa_par > 0.0 || cfg->nu > 0.0 ||
         cfg->eta > 0.0))
        return CTU_EUNSUPPORTED;
    ctu_ctx *ctx = new (std::nothrow) ctu_ctx();
    if (!ctx) return CTU_ENOMEM;
    ctx->cfg = *cfg;
    if (cudaGetDevice(&ctx->device) != cudaSuccess ||
        cudaDeviceGetAttribute(&ctx->sms, cudaDevAttrMultiProcessorCount, ctx->device) != cudaSuccess ||
        cudaMalloc(&ctx->dstatus, sizeof(unsigned int)) != cudaSuccess ||
        cudaMalloc(&ctx->dmax, sizeof(unsigned long long)) != cudaSuccess ||
        cudaMalloc(&ctx->dfloor, sizeof(unsigned long long)) != cudaSuccess ||
        cudaMemset(ctx->dfloor, 0, sizeof(unsigned long long)) != cudaSuccess ||
        cudaMalloc(&ctx->dsp, sizeof(StepParams)) != cudaSuccess ||
        cudaMemset(ctx->dstatus, 0, sizeof(unsigned int)) != cudaSuccess) {
        ctu_destroy(ctx);
        return CTU_ECUDA;
    }
    *out = ctx;
    return CTU_OK;
}

void ctu_destroy(ctu_ctx *ctx)
{
    if (!ctx) return;
    cudaDeviceSynchronize();
    if (ctx->dpatch) cudaFree(ctx->dpatch);
    if (ctx->scratch) cudaFree(ctx->scratch);
    if (ctx->dstatus) cudaFree(ctx->dstatus);
    if (ctx->dmax) cudaFree(ctx->dmax);
    if (ctx->dfloor) cudaFree(ctx->dfloor);
    if (ctx->dtagcnt) cudaFree(ctx->dtagcnt);
    if (ctx->dsp) cudaFree(ctx->dsp);
    if (ctx->dwin) cudaFree(ctx->dwin);
    if (ctx->dwstart) cudaFree(ctx->dwstart);
    for (void *p : ctx->optab)
        if (p) cudaFree(p);
    delete ctx->prof;
    delete ctx;
}

ctu_status ctu_dt(ctu_ctx *ctx, const double *U, int64_t stride, const ctu_patch *patches, int npatch,
                  double *d_dt_ch, double *h_dt_ch, void *stream)
{
    if (!ctx || !U || !d_dt_ch) return CTU_EINVAL;
    ctu_status st = validate_patches(ctx, stride, patches, npatch);
    if (st != CTU_OK) return st;
    cudaStream_t s = (cudaStream_t)stream;
    st = bind_patches(ctx, patches, npatch, s);
    if (st != CTU_OK) return st;
    CTU_CUDA(cudaMemsetAsync(ctx->dmax, 0, sizeof(unsigned long long), s));
    StepArgs a = make_args(ctx, U, nullptr, stride, npatch, nullptr);
    LaunchInfo li = make_info(ctx);
    if (ctx->cfg.precision != CTU_FP64)
        launch_maxspeed<float>(a, li, ctx->dmax, s);
    else
        launch_maxspeed<double>(a, li, ctx->dmax, s);
    k_dt_finalize<<<1, 1, 0, s>>>(ctx->dmax, ctx->cfg.cfl, ctx->dxmin, d_dt_ch);
    CTU_CUDA(cudaGetLastError());
    if (h_dt_ch) {
        CTU_CUDA(cudaMemcpyAsync(h_dt_ch, d_dt_ch, 2 * sizeof(double), cudaMemcpyDeviceToHost, s));
        CTU_CUDA(cudaStreamSynchronize(s));
    }
    return CTU_OK;
}

// Optional floors of the updated state, applied to the interior cells of
// every patch after the step (the library's reading; the paper fixes no
// floor): rho < rho_floor takes rho_floor, then a pressure below p_floor,
// evaluated with that density, is raised to p_floor through E alone.  Every
// operation is an explicitly rounded float64 operation in the order the
// expressions are written (no contraction), so a cell's decision and result
// depend only on its stored state.  One thread per interior cell; one
// atomic per warp counts the cells changed.
constexpr int FLOOR_BLOCK = 256;
__global__ void __launch_bounds__(FLOOR_BLOCK) k_floor(const DevPatch *patches, double *U, long long us, double gm1,
                                                      double p_floor, double rho_floor, unsigned long long *count)
{
    const DevPatch P = patches[blockIdx.y];
    const long long cnt = (long long)P.n[0] * P.n[1] * P.n[2];
    unsigned hits = 0;
    for (long long t = (long long)blockIdx.x * FLOOR_BLOCK + threadIdx.x; t < cnt;
         t += (long long)gridDim.x * FLOOR_BLOCK) {
        const long long row = t / P.n[0];
        const int x = (int)(t - row * P.n[0]);
        const int y = (int)(row % P.n[1]), z = (int)(row / P.n[1]);
        const long long c = P.base + ((long long)(z + P.g[2]) * P.N[1] + (y + P.g[1])) * P.N[0] + (x + P.g[0]);
        double rho = U[c];
        bool hit = false;
        if (rho_floor > 0.0 && rho < rho_floor) {
            rho = rho_floor;
            U[c] = rho;
            hit = true;
        }
        if (p_floor > 0.0) {
            const double m0 = U[us + c], m1 = U[2 * us + c], m2 = U[3 * us + c];
            const double b0 = U[5 * us + c], b1 = U[6 * us + c], b2 = U[7 * us + c];
            const double mm = __dadd_rn(__dadd_rn(__dmul_rn(m0, m0), __dmul_rn(m1, m1)), __dmul_rn(m2, m2));
            const double bb = __dadd_rn(__dadd_rn(__dmul_rn(b0, b0), __dmul_rn(b1, b1)), __dmul_rn(b2, b2));
            const double ek = __ddiv_rn(__dmul_rn(0.5, mm), rho), em = __dmul_rn(0.5, bb);
            const double p = __dmul_rn(gm1, __dsub_rn(__dsub_rn(U[4 * us + c], ek), em));
            if (p < p_floor) {
                U[4 * us + c] = __dadd_rn(__dadd_rn(__ddiv_rn(p_floor, gm1), ek), em);
                hit = true;
            }
        }
        hits += hit;
    }
    for (int o = 16; o > 0; o >>= 1) hits += __shfl_xor_sync(0xffffffffu, hits, o);
    if ((threadIdx.x & 31) == 0 && hits) atomicAdd(count, (unsigned long long)hits);
}

static bool floors_on(const ctu_ctx *ctx) { return ctx->cfg.p_floor > 0.0 || ctx->cfg.rho_floor > 0.0; }

static int launch_floor(ctu_ctx *ctx, double *U, int64_t stride, int npatch, cudaStream_t s)
{
    long long maxc = 0;
    for (const Group &G : ctx->groups) maxc = std::max(maxc, (long long)G.n[0] * G.n[1] * G.n[2]);
    long long bx = (maxc + FLOOR_BLOCK - 1) / FLOOR_BLOCK;
    if (bx > 65535) bx = 65535;
    k_floor<<<dim3((unsigned)bx, (unsigned)npatch, 1), FLOOR_BLOCK, 0, s>>>(
        ctx->dpatch, U, stride, ctx->cfg.gamma - 1.0, ctx->cfg.p_floor, ctx->cfg.rho_floor, ctx->dfloor);
    return 1;
}

static ctu_status step_common(ctu_ctx *ctx, const double *U_in, double *U_out, int64_t stride,
                              const ctu_patch *patches, int npatch, const double *d_dt_ch, double *d_next,
                              void *stream)
{
    if (!ctx || !U_in || !U_out || !d_dt_ch || U_in == U_out) return CTU_EINVAL;
    ctu_status st = validate_patches(ctx, stride, patches, npatch);
    if (st != CTU_OK) return st;
    cudaStream_t s = (cudaStream_t)stream;
    st = bind_patches(ctx, patches, npatch, s);
    if (st != CTU_OK) return st;
    st = ensure_scratch(ctx);
    if (st != CTU_OK) return st;
    StepArgs a = make_args(ctx, U_in, U_out, stride, npatch, d_dt_ch);
    LaunchInfo li = make_info(ctx);
    int n = 0;
    const bool floors = floors_on(ctx);
    if (d_next) {
        CTU_CUDA(cudaMemsetAsync(ctx->dmax, 0, sizeof(unsigned long long), s));
        // with floors, the CFL rate is taken after them, from U_out (with
        // conduction the step's last kernel, the conduction update, reduces
        // it in place of the last sweep)
        if (!floors) a.nextmax = ctx->dmax;
    }
    if (ctx->cfg.precision != CTU_FP64)
        n = launch_step<float>(a, li, s);
    else
        n = launch_step<double>(a, li, s);
    if (floors) {
        n += launch_floor(ctx, U_out, stride, npatch, s);
        if (d_next) {
            StepArgs b = make_args(ctx, U_out, nullptr, stride, npatch, nullptr);
            n += ctx->cfg.precision != CTU_FP64 ? launch_maxspeed<float>(b, li, ctx->dmax, s)
                                                : launch_maxspeed<double>(b, li, ctx->dmax, s);
        }
    }
    if (d_next) {
        k_dt_finalize<<<1, 1, 0, s>>>(ctx->dmax, ctx->cfg.cfl, ctx->dxmin, d_next);
        ++n;
    }
    ctx->last_launches = n;
    CTU_CUDA(cudaGetLastError());
    return CTU_OK;
}

ctu_status ctu_step(ctu_ctx *ctx, const double *U_in, double *U_out, int64_t stride,
                    const ctu_patch *patches, int npatch, const double *d_dt_ch, void *stream)
{
    return step_common(ctx, U_in, U_out, stride, patches, npatch, d_dt_ch, nullptr, stream);
}

ctu_status ctu_step_next_dt(ctu_ctx *ctx, const double *U_in, double *U_out, int64_t stride,
                            const ctu_patch *patches, int npatch, const double *d_dt_ch,
                            double *d_dt_ch_next, void *stream)
{
    if (!d_dt_ch_next || d_dt_ch_next == d_dt_ch) return CTU_EINVAL;
    return step_common(ctx, U_in, U_out, stride, patches, npatch, d_dt_ch, d_dt_ch_next, stream);
}

ctu_status ctu_autotune(ctu_ctx *ctx, const double *U_in, double *U_out, int64_t stride, const ctu_patch *patches,
                        int npatch, const double *d_dt_ch, void *stream)
{
    if (!ctx || !U_in || !U_out || !d_dt_ch || U_in == U_out) return CTU_EINVAL;
    ctu_status st = validate_patches(ctx, stride, patches, npatch);
    if (st != CTU_OK) return st;
    cudaStream_t s = (cudaStream_t)stream;
    st = bind_patches(ctx, patches, npatch, s);
    if (st != CTU_OK) return st;
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    CTU_CUDA(cudaEventCreate(&e0));
    if (cudaEventCreate(&e1) != cudaSuccess) {
        cudaEventDestroy(e0);
        return CTU_ECUDA;
    }
    ctx->tuning = true;
    auto timed = [&](float &ms) -> ctu_status {
        ctu_status r = step_common(ctx, U_in, U_out, stride, patches, npatch, d_dt_ch, nullptr, stream);
        if (r != CTU_OK) return r;
        float best = 1e30f;
        for (int rep = 0; rep < 2; ++rep) {
            if (cudaEventRecord(e0, s) != cudaSuccess) return CTU_ECUDA;
            r = step_common(ctx, U_in, U_out, stride, patches, npatch, d_dt_ch, nullptr, stream);
            if (r != CTU_OK) return r;
            if (cudaEventRecord(e1, s) != cudaSuccess || cudaEventSynchronize(e1) != cudaSuccess) return CTU_ECUDA;
            float t = 0.0f;
            if (cudaEventElapsedTime(&t, e0, e1) != cudaSuccess) return CTU_ECUDA;
            best = std::min(best, t);
        }
        ms = best;
        return CTU_OK;
    };
    // coordinate descent over the shapes, largest first: for each, every
    // (tile width, segment) candidate with the other shapes fixed
    static const int kXw[] = {8, 16, 32};
    static const int kSeg[] = {4, 8, 16, 32, 64};
    for (size_t g = 0; g < ctx->groups.size() && st == CTU_OK; ++g) {
        Group &G = ctx->groups[g];
        int bx = G.xw, bs = G.seg;
        float bt = 1e30f;
        const int nmax = std::max(G.n[0], std::max(G.n[1], G.n[2]));
        for (int xw : kXw) {
            if (xw > 8 && xw / 2 >= G.n[0] + 2) continue;  // wider than the patch
            for (int sg : kSeg) {
                if (sg > 4 && sg / 2 >= nmax) continue;    // longer than any pencil
                G.xw = xw;
                G.seg = sg;
                if (!grid_fits(ctx->groups, ctx->cfg.ndim)) continue;
                float t = 0.0f;
                st = timed(t);
                if (st != CTU_OK) break;
                if (t < bt) {
                    bt = t;
                    bx = xw;
                    bs = sg;
                }
            }
            if (st != CTU_OK) break;
        }
        G.xw = bx;
        G.seg = bs;
        ctx->tune[shape_key(G.n)] = {bx, bs};
    }
    ctx->tuning = false;
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    return st;
}

// ---------------------------------------------------------------- level operators

// Device copy of a descriptor array (kind 0 prolong, 1 restrict, 2 reflux)
// followed by its block map (first block of each descriptor, descriptor of
// each block; blocks[i] = blocks of descriptor i), uploaded only when the
// descriptors change.
static ctu_status ensure_tag_scratch(ctu_ctx *ctx, int npatch)
{
    if (npatch <= ctx->dtagcnt_cap) return CTU_OK;
    CTU_CUDA(cudaDeviceSynchronize());
    if (ctx->dtagcnt) cudaFree(ctx->dtagcnt);
    ctx->dtagcnt = nullptr;
    ctx->dtagcnt_cap = 0;
    CTU_CUDA(cudaMalloc(&ctx->dtagcnt, sizeof(unsigned long long) * npatch));
    ctx->dtagcnt_cap = npatch;
    return CTU_OK;
}

struct OpTable {
    const void *desc;
    BlockMap map;
    unsigned nblocks;
};

static ctu_status op_table(ctu_ctx *ctx, int kind, const void *h, size_t bytes, int n, const long long *blocks,
                           cudaStream_t s, OpTable *out)
{
    std::vector<char> &c = ctx->opcache[kind];
    long long tot = 0;
    for (int i = 0; i < n; ++i) tot += blocks[i];
    if (tot >= (1LL << 31)) return CTU_EINVAL;
    const size_t dbytes = (bytes + 15) / 16 * 16;
    const size_t need = dbytes + sizeof(int) * ((size_t)n + (size_t)tot);
    if (c.size() != bytes || std::memcmp(c.data(), h, bytes) != 0) {
        std::vector<char> img(need);
        std::memcpy(img.data(), h, bytes);
        int *start = (int *)(img.data() + dbytes), *blk = start + n;
        long long b = 0;
        for (int i = 0; i < n; ++i) {
            start[i] = (int)b;
            for (long long k = 0; k < blocks[i]; ++k) blk[b + k] = i;
            b += blocks[i];
        }
        CTU_CUDA(cudaStreamSynchronize(s));
        if (need > ctx->opcap[kind]) {
            if (ctx->optab[kind]) cudaFree(ctx->optab[kind]);
            ctx->optab[kind] = nullptr;
            ctx->opcap[kind] = 0;
            CTU_CUDA(cudaMalloc(&ctx->optab[kind], need));
            ctx->opcap[kind] = need;
        }
        CTU_CUDA(cudaMemcpyAsync(ctx->optab[kind], img.data(), need, cudaMemcpyHostToDevice, s));
        CTU_CUDA(cudaStreamSynchronize(s));
        c.assign((const char *)h, (const char *)h + bytes);
    }
    char *base = (char *)ctx->optab[kind];
    out->desc = base;
    out->map.box_start = (const int *)(base + dbytes);
    out->map.blk_box = out->map.box_start + n;
    out->nblocks = (unsigned)tot;
    return CTU_OK;
}

// Ghosted extent of a patch with n interior cells; false if n is invalid.
static bool patch_extent(const ctu_ctx *ctx, const int n[3], long long *cells)
{
    long long c = 1;
    for (int d = 0; d < 3; ++d) {
        if (d < ctx->cfg.ndim) {
            if (n[d] < 1 || n[d] > (1 << 20)) return false;
            c *= n[d] + 2 * AMR_NG;
        } else if (n[d] != 1) {
            return false;
        }
    }
    *cells = c;
    return true;
}

static int floordiv_h(int a, int b) { return a >= 0 ? a / b : -((-a + b - 1) / b); }

// A level box is valid: both patches inside their pools, the box inside the
// output patch's ghosted region, and every cell it reads inside the input
// patch's ghosted region (prolongation: the coarse cell and its neighbours
// along active dimensions; restriction: all fine children).
static bool box_ok(const ctu_ctx *ctx, const ctu_level_box &B, int64_t cstride, int64_t fstride, bool prolong,
                   long long *cells)
{
    long long cc = 0, fc = 0;
    if (!patch_extent(ctx, B.cn, &cc) || !patch_extent(ctx, B.fn, &fc) || B.ratio < 1 || B.ratio > 4) return false;
    if (B.phys < 0 || B.phys > 63) return false;
    if (B.cbase < 0 || B.cbase + cc > cstride || B.fbase < 0 || B.fbase + fc > fstride) return false;
    const int *out_n = prolong ? B.fn : B.cn;
    long long cnt = 1;
    for (int d = 0; d < 3; ++d) {
        const bool act = d < ctx->cfg.ndim;
        const int g = act ? AMR_NG : 0;
        if (B.hi[d] < B.lo[d]) return false;
        cnt *= B.hi[d] - B.lo[d];
        if (B.hi[d] == B.lo[d]) continue;
        if (!act) {
            if (B.lo[d] != 0 || B.hi[d] != 1) return false;
            continue;
        }
        if (B.lo[d] < -g || B.hi[d] > out_n[d] + g) return false;
        if (prolong) {  // coarse cells origin + floor(x / r) and their neighbours
            const int cmin = B.origin[d] + floordiv_h(B.lo[d], B.ratio) - 1;
            const int cmax = B.origin[d] + floordiv_h(B.hi[d] - 1, B.ratio) + 1;
            if (cmin < -g || cmax >= B.cn[d] + g) return false;
        } else {  // fine children (c - origin) r + k
            const long long fmin = (long long)(B.lo[d] - B.origin[d]) * B.ratio;
            const long long fmax = (long long)(B.hi[d] - 1 - B.origin[d]) * B.ratio + B.ratio - 1;
            if (fmin < -g || fmax >= B.fn[d] + g) return false;
        }
    }
    *cells = cnt;
    return true;
}

ctu_status ctu_prolong(ctu_ctx *ctx, const double *Uc_old, const double *Uc_new, int64_t cstride, double alpha,
                       double *Uf, int64_t fstride, const ctu_level_box *boxes, int nbox, void *stream)
{
    if (!ctx || !Uc_old || !Uc_new || !Uf || !boxes || nbox <= 0 || nbox > 65535 || !(alpha == alpha))
        return CTU_EINVAL;
    if (Uf == Uc_old || Uf == Uc_new) return CTU_EINVAL;
    std::vector<long long> blocks(nbox);
    for (int i = 0; i < nbox; ++i) {
        long long c = 0;
        if (!box_ok(ctx, boxes[i], cstride, fstride, true, &c)) return CTU_EINVAL;
        // one thread per variable and coarse cell under the box, indexed in
        // 32 bits
        long long cc = c > 0 ? 1 : 0;
        for (int d = 0; d < ctx->cfg.ndim && cc; ++d) {
            const ctu_level_box &B = boxes[i];
            cc *= floordiv_h(B.hi[d] - 1, B.ratio) + 1 - floordiv_h(B.lo[d], B.ratio);
        }
        if (9 * cc >= (1LL << 31)) return CTU_EINVAL;
        blocks[i] = (9 * cc + AMR_BLOCK - 1) / AMR_BLOCK;
    }
    cudaStream_t s = (cudaStream_t)stream;
    OpTable T;
    ctu_status st = op_table(ctx, 0, boxes, sizeof(ctu_level_box) * nbox, nbox, blocks.data(), s, &T);
    if (st != CTU_OK) return st;
    if (T.nblocks == 0) return CTU_OK;
    if (ctx->prof) ctx->prof->mark("prolong", s);
    if (alpha == 0.0 || alpha == 1.0)  // U* is one of the two states: no blend
        k_prolong<false><<<T.nblocks, AMR_BLOCK, 0, s>>>((const ctu_level_box *)T.desc, T.map, ctx->cfg.ndim,
                                                         alpha == 0.0 ? Uc_old : Uc_new,
                                                         alpha == 0.0 ? Uc_old : Uc_new, cstride, alpha, Uf, fstride);
    else
        k_prolong<true><<<T.nblocks, AMR_BLOCK, 0, s>>>((const ctu_level_box *)T.desc, T.map, ctx->cfg.ndim,
                                                        Uc_old, Uc_new, cstride, alpha, Uf, fstride);
    if (ctx->prof) ctx->prof->mark(nullptr, s);
    CTU_CUDA(cudaGetLastError());
    return CTU_OK;
}

ctu_status ctu_restrict(ctu_ctx *ctx, double *Uc, int64_t cstride, const double *Uf, int64_t fstride,
                        const ctu_level_box *boxes, int nbox, void *stream)
{
    if (!ctx || !Uc || !Uf || !boxes || nbox <= 0 || nbox > 65535 || Uc == Uf) return CTU_EINVAL;
    std::vector<long long> blocks(nbox);
    for (int i = 0; i < nbox; ++i) {
        long long c = 0;
        if (!box_ok(ctx, boxes[i], cstride, fstride, false, &c)) return CTU_EINVAL;
        // one thread per coarse cell, indexed in 32 bits
        if (c >= (1LL << 31)) return CTU_EINVAL;
        blocks[i] = (c + AMR_BLOCK - 1) / AMR_BLOCK;
    }
    cudaStream_t s = (cudaStream_t)stream;
    OpTable T;
    ctu_status st = op_table(ctx, 1, boxes, sizeof(ctu_level_box) * nbox, nbox, blocks.data(), s, &T);
    if (st != CTU_OK) return st;
    if (T.nblocks == 0) return CTU_OK;
    if (ctx->prof) ctx->prof->mark("restrict", s);
    k_restrict<<<T.nblocks, AMR_BLOCK, 0, s>>>((const ctu_level_box *)T.desc, T.map, ctx->cfg.ndim, Uc, cstride,
                                              Uf, fstride);
    if (ctx->prof) ctx->prof->mark(nullptr, s);
    CTU_CUDA(cudaGetLastError());
    return CTU_OK;
}

ctu_status ctu_reflux(ctu_ctx *ctx, double *Uc, int64_t cstride, const double *reg, const ctu_reflux_set *sets,
                      int nset, void *stream)
{
    if (!ctx || !Uc || !reg || !sets || nset <= 0 || nset > 65535) return CTU_EINVAL;
    const int ndim = ctx->cfg.ndim;
    // sets ordered by class (direction, then side), one launch per class
    auto cls = [](const ctu_reflux_set &S) { return 2 * S.dir + (S.side > 0 ? 1 : 0); };
    std::vector<ctu_reflux_set> ord(sets, sets + nset);
    std::stable_sort(ord.begin(), ord.end(),
                     [&](const ctu_reflux_set &x, const ctu_reflux_set &y) { return cls(x) < cls(y); });
    std::vector<long long> blocks(nset);
    long long cblk[7] = {0, 0, 0, 0, 0, 0, 0};
    for (int i = 0; i < nset; ++i) {
        const ctu_reflux_set &S = ord[i];
        long long cc = 0;
        if (!patch_extent(ctx, S.cn, &cc) || S.cbase < 0 || S.cbase + cc > cstride) return CTU_EINVAL;
        if (S.dir < 0 || S.dir >= ndim || (S.side != 1 && S.side != -1) || S.ratio < 1) return CTU_EINVAL;
        const int cell = S.side > 0 ? S.plane : S.plane - 1;
        if (cell < 0 || cell >= S.cn[S.dir]) return CTU_EINVAL;
        const int ea = S.dir == 0 ? 1 : 0, eb = S.dir == 2 ? 1 : 2;
        if (S.a0 < 0 || S.a1 < S.a0 || S.a1 > S.cn[ea] || S.b0 < 0 || S.b1 < S.b0 || S.b1 > S.cn[eb]) return CTU_EINVAL;
        if (S.creg < 0 || S.freg < 0 || S.fa0 < 0 || S.fb0 < 0 || S.fna < 0 || S.fnb < 0) return CTU_EINVAL;
        const long long ra = ea < ndim ? S.ratio : 1, rb = eb < ndim ? S.ratio : 1;
        if (S.a1 > S.a0 && S.b1 > S.b0 &&
            (S.fa0 + (S.a1 - S.a0) * ra > S.fna || S.fb0 + (S.b1 - S.b0) * rb > S.fnb))
            return CTU_EINVAL;
        for (int d = 0; d < ndim; ++d)
            if (!(S.dx[d] > 0.0)) return CTU_EINVAL;
        // one thread per variable and coarse face, indexed in 32 bits
        const long long nf = 9LL * (S.a1 - S.a0) * (S.b1 - S.b0);
        if (nf >= (1LL << 31)) return CTU_EINVAL;
        blocks[i] = (nf + AMR_BLOCK - 1) / AMR_BLOCK;
        cblk[cls(S) + 1] += blocks[i];
    }
    cudaStream_t s = (cudaStream_t)stream;
    OpTable T;
    ctu_status st = op_table(ctx, 2, ord.data(), sizeof(ctu_reflux_set) * nset, nset, blocks.data(), s, &T);
    if (st != CTU_OK) return st;
    if (T.nblocks == 0) return CTU_OK;
    if (ctx->prof) ctx->prof->mark("reflux", s);
    long long b0 = 0;
    for (int c = 0; c < 6; ++c) {
        if (cblk[c + 1] > 0)
            k_reflux<<<(unsigned)cblk[c + 1], AMR_BLOCK, 0, s>>>((const ctu_reflux_set *)T.desc, T.map, (unsigned)b0,
                                                               ndim, Uc, cstride, reg);
        b0 += cblk[c + 1];
    }
    if (ctx->prof) ctx->prof->mark(nullptr, s);
    CTU_CUDA(cudaGetLastError());
    return CTU_OK;
}

}  // extern "C"

template <int K>
static void launch_tag(const OpTable &T, TagArgs a, bool tile, cudaStream_t s)
{
    a.tp = (const TagPatch *)T.desc;
    a.map = T.map;
    if (tile)
        k_tag_tile<K><<<T.nblocks, TAG_TILE, 0, s>>>(a);
    else if (a.chi)
        k_tag_flat<K, true><<<T.nblocks, AMR_BLOCK, 0, s>>>(a);
    else
        k_tag_flat<K, false><<<T.nblocks, AMR_BLOCK, 0, s>>>(a);
}

extern "C" {

ctu_status ctu_tag(ctu_ctx *ctx, const double *U, int64_t stride, const ctu_patch *patches, int npatch, int sigma,
                   double eps, double chi_r, unsigned char *tags, int64_t *d_count, double *chi, void *stream)
{
    if (!ctx || !U || !tags || !patches || npatch <= 0) return CTU_EINVAL;
    if (sigma < CTU_TAG_DENSITY || sigma > CTU_TAG_E_OVER_RHO) return CTU_EINVAL;
    if (!(eps >= 0.0 && eps < INFINITY) || !(chi_r >= 0.0 && chi_r < INFINITY)) return CTU_EINVAL;
    ctu_status st = validate_patches(ctx, stride, patches, npatch);
    if (st != CTU_OK) return st;
    // patches of a plane width >= 16 in 2-D and 3-D march in tiles; the rest
    // (and every patch when chi is written) take one cell per thread
    std::vector<TagPatch> tp[2];
    std::vector<long long> blocks[2];
    const int nd = ctx->cfg.ndim;
    for (int i = 0; i < npatch; ++i) {
        TagPatch q;
        for (int d = 0; d < 3; ++d) q.n[d] = patches[i].n[d];
        q.slot = i;
        q.base = patches[i].base;
        const bool tile = !chi && nd >= 2 && q.n[0] >= 16;
        const long long b = tile ? (long long)((q.n[0] + TAG_TX - 1) / TAG_TX) * ((q.n[1] + TAG_TY - 1) / TAG_TY) *
                                       ((q.n[2] + TAG_SZ - 1) / TAG_SZ)
                                 : ((long long)q.n[0] * q.n[1] * q.n[2] + AMR_BLOCK - 1) / AMR_BLOCK;
        tp[tile].push_back(q);
        blocks[tile].push_back(b);
    }
    cudaStream_t s = (cudaStream_t)stream;
    // per-patch counts: the caller's array, else the context's scratch
    unsigned long long *cnt = (unsigned long long *)d_count;
    if (!cnt) {
        st = ensure_tag_scratch(ctx, npatch);
        if (st != CTU_OK) return st;
        cnt = ctx->dtagcnt;
    }
    OpTable T[2];
    for (int g = 0; g < 2; ++g) {
        T[g].nblocks = 0;
        if (tp[g].empty()) continue;
        st = op_table(ctx, 3 + g, tp[g].data(), sizeof(TagPatch) * tp[g].size(), (int)tp[g].size(),
                      blocks[g].data(), s, &T[g]);
        if (st != CTU_OK) return st;
    }
    CTU_CUDA(cudaMemsetAsync(cnt, 0, sizeof(unsigned long long) * npatch, s));
    const double f = tag_margin(sigma, eps, chi_r);
    TagArgs a;
    a.ndim = nd;
    a.U = U;
    a.us = stride;
    a.eps = eps;
    a.chi_r = chi_r;
    a.eps32 = (float)eps;
    a.c2 = (float)(chi_r * chi_r);
    a.filt = f < 1.0 ? (float)f : INFINITY;
    a.tags = tags;
    a.counts = cnt;
    a.chi = chi;
    if (ctx->prof) ctx->prof->mark("tag", s);
    int launches = 0;
    for (int g = 0; g < 2; ++g) {
        if (T[g].nblocks == 0) continue;
        switch (sigma) {
        case CTU_TAG_DENSITY: launch_tag<0>(T[g], a, g == 1, s); break;
        case CTU_TAG_ENERGY: launch_tag<1>(T[g], a, g == 1, s); break;
        case CTU_TAG_B2_OVER_RHO: launch_tag<2>(T[g], a, g == 1, s); break;
        default: launch_tag<3>(T[g], a, g == 1, s); break;
        }
        ++launches;
    }
    if (ctx->prof) ctx->prof->mark(nullptr, s);
    ctx->last_launches = launches;
    CTU_CUDA(cudaGetLastError());
    return CTU_OK;
}

// Checks every box against its patches and pools (mode 0 both sides, 1 the
// source, 2 the destination) and builds the device descriptors.
static ctu_status copy_table(ctu_ctx *ctx, int mode, const ctu_copy_box *boxes, int nbox, int64_t dstride,
                             int64_t sstride, cudaStream_t s, OpTable *T)
{
    if (!boxes || nbox <= 0 || nbox > (1 << 24)) return CTU_EINVAL;
    const int nd = ctx->cfg.ndim;
    std::vector<CopyDesc> D(nbox);
    std::vector<long long> blocks(nbox);
    long long off = 0;
    for (int i = 0; i < nbox; ++i) {
        const ctu_copy_box &b = boxes[i];
        CopyDesc &c = D[i];
        long long cells = 1, dc = 0, sc = 0;
        for (int d = 0; d < 3; ++d) {
            c.dn[d] = b.dn[d];
            c.sn[d] = b.sn[d];
            c.lo[d] = b.lo[d];
            c.ext[d] = b.hi[d] - b.lo[d];
            c.shift[d] = b.shift[d];
            if (c.ext[d] < 1) return CTU_EINVAL;
            cells *= c.ext[d];
            const int g = d < nd ? 4 : 0;
            if (mode != 1) {
                if (b.dn[d] < 1 || (d >= nd && b.dn[d] != 1) || b.lo[d] < -g || b.hi[d] > b.dn[d] + g) return CTU_EINVAL;
            }
            if (mode != 2) {
                if (b.sn[d] < 1 || (d >= nd && b.sn[d] != 1) || b.lo[d] + b.shift[d] < -g ||
                    b.hi[d] + b.shift[d] > b.sn[d] + g)
                    return CTU_EINVAL;
            }
        }
        if (cells >= (1LL << 31)) return CTU_EINVAL;
        c.pad = 0;
        c.dbase = b.dbase;
        c.sbase = b.sbase;
        c.boff = off;
        off += 9 * cells;
        if (mode != 1) {
            if (!patch_extent(ctx, b.dn, &dc) || b.dbase < 0 || b.dbase + dc > dstride) return CTU_EINVAL;
        }
        if (mode != 2) {
            if (!patch_extent(ctx, b.sn, &sc) || b.sbase < 0 || b.sbase + sc > sstride) return CTU_EINVAL;
        }
        blocks[i] = (cells + AMR_BLOCK - 1) / AMR_BLOCK;
    }
    return op_table(ctx, 5 + mode, D.data(), sizeof(CopyDesc) * nbox, nbox, blocks.data(), s, T);
}

ctu_status ctu_copy(ctu_ctx *ctx, double *U_dst, int64_t dstride, const double *U_src, int64_t sstride,
                    const ctu_copy_box *boxes, int nbox, void *stream)
{
    if (!ctx || !U_dst || !U_src) return CTU_EINVAL;
    cudaStream_t s = (cudaStream_t)stream;
    OpTable T;
    ctu_status st = copy_table(ctx, 0, boxes, nbox, dstride, sstride, s, &T);
    if (st != CTU_OK) return st;
    if (ctx->prof) ctx->prof->mark("exchange", s);
    k_copy<0><<<T.nblocks, AMR_BLOCK, 0, s>>>((const CopyDesc *)T.desc, T.map, ctx->cfg.ndim, U_dst, dstride, U_src,
                                             sstride);
    if (ctx->prof) ctx->prof->mark(nullptr, s);
    CTU_CUDA(cudaGetLastError());
    return CTU_OK;
}

ctu_status ctu_pack(ctu_ctx *ctx, double *buf, const double *U_src, int64_t sstride, const ctu_copy_box *boxes,
                    int nbox, void *stream)
{
    if (!ctx || !buf || !U_src) return CTU_EINVAL;
    cudaStream_t s = (cudaStream_t)stream;
    OpTable T;
    ctu_status st = copy_table(ctx, 1, boxes, nbox, 0, sstride, s, &T);
    if (st != CTU_OK) return st;
    k_copy<1><<<T.nblocks, AMR_BLOCK, 0, s>>>((const CopyDesc *)T.desc, T.map, ctx->cfg.ndim, buf, 0, U_src,
                                             sstride);
    CTU_CUDA(cudaGetLastError());
    return CTU_OK;
}

ctu_status ctu_unpack(ctu_ctx *ctx, double *U_dst, int64_t dstride, const double *buf, const ctu_copy_box *boxes,
                      int nbox, void *stream)
{
    if (!ctx || !buf || !U_dst) return CTU_EINVAL;
    cudaStream_t s = (cudaStream_t)stream;
    OpTable T;
    ctu_status st = copy_table(ctx, 2, boxes, nbox, dstride, 0, s, &T);
    if (st != CTU_OK) return st;
    k_copy<2><<<T.nblocks, AMR_BLOCK, 0, s>>>((const CopyDesc *)T.desc, T.map, ctx->cfg.ndim, U_dst, dstride, buf,
                                             0);
    CTU_CUDA(cudaGetLastError());
    return CTU_OK;
}

ctu_status ctu_diagnostics(ctu_ctx *ctx, const double *U, int64_t stride, const ctu_patch *patches, int npatch,
                           double *d_out, void *stream)
{
    if (!ctx || !U || !d_out) return CTU_EINVAL;
    ctu_status st = validate_patches(ctx, stride, patches, npatch);
    if (st != CTU_OK) return st;
    cudaStream_t s = (cudaStream_t)stream;
    st = bind_patches(ctx, patches, npatch, s);
    if (st != CTU_OK) return st;
    long long maxc = 0;
    for (const Group &G : ctx->groups) maxc = std::max(maxc, (long long)G.n[0] * G.n[1] * G.n[2]);
    long long bx = (maxc + AMR_BLOCK - 1) / AMR_BLOCK;
    if (bx > 1024) bx = 1024;
    CTU_CUDA(cudaMemsetAsync(d_out, 0, 10 * sizeof(double), s));
    k_diagnostics<<<dim3((unsigned)bx, (unsigned)npatch), AMR_BLOCK, 0, s>>>(ctx->dpatch, ctx->cfg.ndim, U, stride,
                                                                             d_out);
    CTU_CUDA(cudaGetLastError());
    return CTU_OK;
}

ctu_status ctu_tile_params(ctu_ctx *ctx, const int n[3], int *xw, int *seg)
{
    if (!ctx || !n || !xw || !seg) return CTU_EINVAL;
    const auto it = ctx->tune.find(shape_key(n));
    *xw = it != ctx->tune.end() ? it->second[0] : Tiles::xw(n[0]);
    *seg = it != ctx->tune.end() ? it->second[1] : SEG;
    return CTU_OK;
}

ctu_status ctu_flux_registers(ctu_ctx *ctx, double *reg, const ctu_flux_window *win, int nwin)
{
    if (!ctx || nwin < 0) return CTU_EINVAL;
    if (!reg || nwin == 0) {
        ctx->reg = nullptr;
        ctx->hwin.clear();
        ctx->win_dirty = false;
        return CTU_OK;
    }
    if (!win) return CTU_EINVAL;
    for (int i = 0; i < nwin; ++i) {
        const ctu_flux_window &x = win[i];
        if (x.patch < 0 || x.dir < 0 || x.dir >= ctx->cfg.ndim || x.a1 < x.a0 || x.b1 < x.b0 || x.a0 < 0 ||
            x.b0 < 0 || x.dst < 0 || x.plane < 0)
            return CTU_EINVAL;
    }
    CTU_CUDA(cudaDeviceSynchronize());
    ctx->hwin.assign(win, win + nwin);
    ctx->reg = reg;
    ctx->win_dirty = true;
    if (!ctx->hpatch.empty()) return upload_windows(ctx, 0);
    return CTU_OK;
}

__global__ void k_fill_periodic(const DevPatch *patches, int ndim, double *U, long long stride)
{
    const DevPatch P = patches[blockIdx.y];
    const long long ncell = (long long)P.N[0] * P.N[1] * P.N[2];
    for (long long c = blockIdx.x * (long long)blockDim.x + threadIdx.x; c < ncell;
         c += (long long)gridDim.x * blockDim.x) {
        int x[3];
        x[0] = (int)(c % P.N[0]) - P.g[0];
        x[1] = (int)((c / P.N[0]) % P.N[1]) - P.g[1];
        x[2] = (int)(c / ((long long)P.N[0] * P.N[1])) - P.g[2];
        bool ghost = false;
        int y[3];
        for (int d = 0; d < 3; ++d) {
            y[d] = x[d];
            if (d < ndim && (x[d] < 0 || x[d] >= P.n[d])) {
                ghost = true;
                y[d] = ((x[d] % P.n[d]) + P.n[d]) % P.n[d];
            }
        }
        if (!ghost) continue;
        const long long src = ((long long)(y[2] + P.g[2]) * P.N[1] + (y[1] + P.g[1])) * P.N[0] + (y[0] + P.g[0]);
        for (int q = 0; q < NV; ++q) U[q * stride + P.base + c] = U[q * stride + P.base + src];
    }
}

ctu_status ctu_fill_periodic(ctu_ctx *ctx, double *U, int64_t stride, const ctu_patch *patches, int npatch,
                             void *stream)
{
    if (!ctx || !U) return CTU_EINVAL;
    ctu_status st = validate_patches(ctx, stride, patches, npatch);
    if (st != CTU_OK) return st;
    cudaStream_t s = (cudaStream_t)stream;
    st = bind_patches(ctx, patches, npatch, s);
    if (st != CTU_OK) return st;
    long long maxc = 0;
    for (const Group &G : ctx->groups) maxc = std::max(maxc, (long long)G.N[0] * G.N[1] * G.N[2]);
    long long bx = (maxc + 255) / 256;
    if (bx > (1LL << 20)) bx = 1LL << 20;
    k_fill_periodic<<<dim3((unsigned)bx, (unsigned)npatch, 1), 256, 0, s>>>(ctx->dpatch, ctx->cfg.ndim, U, stride);
    CTU_CUDA(cudaGetLastError());
    return CTU_OK;
}

ctu_status ctu_floor_count(ctu_ctx *ctx, int64_t *count, void *stream)
{
    if (!ctx || !count) return CTU_EINVAL;
    cudaStream_t s = (cudaStream_t)stream;
    unsigned long long h = 0;
    CTU_CUDA(cudaStreamSynchronize(s));
    CTU_CUDA(cudaMemcpy(&h, ctx->dfloor, sizeof(h), cudaMemcpyDeviceToHost));
    CTU_CUDA(cudaMemset(ctx->dfloor, 0, sizeof(h)));
    *count = (int64_t)h;
    return CTU_OK;
}

ctu_status ctu_status_sync(ctu_ctx *ctx, void *stream)
{
    if (!ctx) return CTU_EINVAL;
    cudaStream_t s = (cudaStream_t)stream;
    unsigned int h = 0;
    CTU_CUDA(cudaStreamSynchronize(s));
    CTU_CUDA(cudaMemcpy(&h, ctx->dstatus, sizeof(h), cudaMemcpyDeviceToHost));
    CTU_CUDA(cudaMemset(ctx->dstatus, 0, sizeof(unsigned int)));
    if (h & ST_NAN) return CTU_ENAN;
    if (h & ST_REC) return CTU_ERECOVERY;
    if (h & ST_SUPER) return CTU_ESUPERLUMINAL;
    if (h & ST_NEG) return CTU_ENEGATIVE;
    return CTU_OK;
}

const char *ctu_strerror(ctu_status s)
{
    switch (s) {
    case CTU_OK: return "ok";
    case CTU_EINVAL: return "invalid argument";
    case CTU_ENOMEM: return "out of memory";
    case CTU_ECUDA: return "CUDA runtime error";
    case CTU_EUNSUPPORTED: return "unsupported configuration";
    case CTU_ENEGATIVE: return "non-positive density or pressure met";
    case CTU_ENAN: return "NaN or Inf met";
    case CTU_ERECOVERY: return "primitive recovery did not converge";
    case CTU_ESUPERLUMINAL: return "superluminal velocity met";
    case CTU_ETIMEOUT: return "bounded wait timed out";
    case CTU_ETOOLARGE: return "batch exceeds the fixed scratch of ctu_step_noalloc";
    }
    return "unknown status";
}

int ctu_last_launch_count(const ctu_ctx *ctx) { return ctx ? ctx->last_launches : -1; }

ctu_status ctu_profile(ctu_ctx *ctx, int enable)
{
    if (!ctx) return CTU_EINVAL;
    CTU_CUDA(cudaDeviceSynchronize());
    if (!enable) {
        delete ctx->prof;
        ctx->prof = nullptr;
        return CTU_OK;
    }
    if (!ctx->prof) ctx->prof = new (std::nothrow) EventProf();
    if (!ctx->prof) return CTU_ENOMEM;
    ctx->prof->reset();
    return CTU_OK;
}

int ctu_profile_read(ctu_ctx *ctx, int i, const char **name, double *total_ms, long long *launches)
{
    if (!ctx || !ctx->prof) return 0;
    if (cudaDeviceSynchronize() != cudaSuccess) return 0;
    ctx->prof->resolve();
    const int n = (int)ctx->prof->names.size();
    if (i >= 0 && i < n) {
        const std::string &k = ctx->prof->names[i];
        const auto &v = ctx->prof->tot[k];
        if (name) *name = k.c_str();
        if (total_ms) *total_ms = v.first;
        if (launches) *launches = v.second;
    }
    return n;
}

} // extern "C"
