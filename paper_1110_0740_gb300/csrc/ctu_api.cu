// ctu_api.cu -- C ABI of libctu.so (declared in include/ctu.h).
//
// Host side of the CTU-MHD integrator: argument validation, patch-list
// upload, scratch management, the CFL reduction of Eq. (Ca), the step
// launch sequence, flux-register binding and the sticky device status.
#include <cuda_runtime.h>

#include <cstdint>
#include <cstdlib>
#include <cstring>
#include <map>
#include <new>
#include <string>
#include <vector>

#include "ctu.h"
#include "ctu_launch.h"

using namespace ctu;

// Per-kernel CUDA-event timing: an event is recorded on the launching stream
// right before and right after every kernel; totals are resolved on read.
struct EventProf : ProfHook {
    struct Rec { const char *name; cudaEvent_t a, b; };
    std::vector<cudaEvent_t> pool;
    size_t used = 0;
    std::vector<Rec> pending;
    const char *open = nullptr;
    cudaEvent_t open_ev = nullptr;
    std::vector<std::string> names;
    std::map<std::string, std::pair<double, long>> tot;
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
                auto it = tot.find(r.name);
                if (it == tot.end()) {
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

struct ctu_ctx {
    ctu_config cfg;
    int device = 0;
    // patch list cache
    std::vector<ctu_patch> hpatch;
    DevPatch *dpatch = nullptr;
    int dpatch_cap = 0;
    long long sstride = 0;
    long long max_cells = 0;
    long long max_interior = 0;
    double dxmin = 0.0;
    // scratch
    void *scratch = nullptr;
    size_t scratch_bytes = 0;
    // status, reduction word
    unsigned int *dstatus = nullptr;
    unsigned long long *dmax = nullptr;
    // flux registers
    DevWindow *dwin = nullptr;
    int nwin = 0;
    double *reg = nullptr;
    int last_launches = 0;
    EventProf *prof = nullptr;
};

static ctu_status cuda_fail(cudaError_t e)
{
    return e == cudaErrorMemoryAllocation ? CTU_ENOMEM : CTU_ECUDA;
}

#define CTU_CUDA(call)                                    \
    do {                                                  \
        cudaError_t e_ = (call);                          \
        if (e_ != cudaSuccess) return cuda_fail(e_);      \
    } while (0)

static int active_ghost(const ctu_ctx *ctx, int d) { return d < ctx->cfg.ndim ? 4 : 0; }

static ctu_status validate_patches(const ctu_ctx *ctx, int64_t stride, const ctu_patch *p, int np)
{
    if (!p || np <= 0 || np > 65535) return CTU_EINVAL;
    for (int i = 0; i < np; ++i) {
        long long cells = 1;
        for (int d = 0; d < 3; ++d) {
            if (p[i].n[d] < 1) return CTU_EINVAL;
            if (d >= ctx->cfg.ndim && p[i].n[d] != 1) return CTU_EINVAL;
            if (!(p[i].dx[d] > 0.0)) return CTU_EINVAL;
            cells *= (long long)p[i].n[d] + 2 * active_ghost(ctx, d);
        }
        if (p[i].base < 0 || p[i].base + cells > stride) return CTU_EINVAL;
    }
    return CTU_OK;
}

// Upload the patch list if it differs from the cached one; sizes scratch.
static ctu_status bind_patches(ctu_ctx *ctx, const ctu_patch *p, int np, cudaStream_t s)
{
    if ((int)ctx->hpatch.size() == np && std::memcmp(ctx->hpatch.data(), p, sizeof(ctu_patch) * np) == 0)
        return CTU_OK;
    std::vector<DevPatch> dp(np);
    long long off = 0, maxc = 0, maxi = 0;
    double dxmin = 1e300;
    for (int i = 0; i < np; ++i) {
        DevPatch &q = dp[i];
        long long cells = 1, inner = 1;
        for (int d = 0; d < 3; ++d) {
            q.n[d] = p[i].n[d];
            q.g[d] = active_ghost(ctx, d);
            q.N[d] = q.n[d] + 2 * q.g[d];
            q.dx[d] = p[i].dx[d];
            cells *= q.N[d];
            inner *= q.n[d];
            if (d < ctx->cfg.ndim && q.dx[d] < dxmin) dxmin = q.dx[d];
        }
        q.base = p[i].base;
        q.soff = off;
        off += (cells + 31) / 32 * 32;
        if (cells > maxc) maxc = cells;
        if (inner > maxi) maxi = inner;
    }
    if (np > ctx->dpatch_cap) {
        if (ctx->dpatch) cudaFree(ctx->dpatch);
        ctx->dpatch = nullptr;
        CTU_CUDA(cudaMalloc(&ctx->dpatch, sizeof(DevPatch) * np));
        ctx->dpatch_cap = np;
    }
    CTU_CUDA(cudaMemcpyAsync(ctx->dpatch, dp.data(), sizeof(DevPatch) * np, cudaMemcpyHostToDevice, s));
    CTU_CUDA(cudaStreamSynchronize(s));
    ctx->hpatch.assign(p, p + np);
    ctx->sstride = off;
    ctx->max_cells = maxc;
    ctx->max_interior = maxi;
    ctx->dxmin = dxmin;
    return CTU_OK;
}

static ctu_status ensure_scratch(ctu_ctx *ctx)
{
    const size_t elt = ctx->cfg.precision == CTU_FP64 ? sizeof(double) : sizeof(float);
    const size_t need = (size_t)SCRATCH_ARRAYS * (size_t)ctx->sstride * elt;
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
    a.patches = ctx->dpatch;
    a.npatch = np;
    a.ndim = ctx->cfg.ndim;
    a.gam = ctx->cfg.gamma;
    a.glm_alpha = ctx->cfg.glm_alpha;
    a.upwind = ctx->cfg.trace_mode == CTU_TRACE_UPWIND;
    a.U = Uin;
    a.Uout = Uout;
    a.ustride = stride;
    a.sstride = ctx->sstride;
    a.dtch = dtch;
    a.status = ctx->dstatus;
    return a;
}

extern "C" {

ctu_status ctu_init(const ctu_config *cfg, ctu_ctx **out)
{
    if (!cfg || !out) return CTU_EINVAL;
    *out = nullptr;
    if (cfg->physics != CTU_MHD) return cfg->physics == CTU_SRMHD ? CTU_EUNSUPPORTED : CTU_EINVAL;
    if (cfg->eos != CTU_EOS_IDEAL) return CTU_EUNSUPPORTED;
    if (!(cfg->gamma > 1.0)) return CTU_EINVAL;
    if (cfg->ndim < 1 || cfg->ndim > 3) return CTU_EINVAL;
    if (cfg->recon != CTU_LINEAR_MC && cfg->recon != CTU_PPM) return CTU_EINVAL;
    if (cfg->predictor != CTU_CHAR_TRACE) return CTU_EUNSUPPORTED;
    if (cfg->riemann != CTU_HLLD) return CTU_EUNSUPPORTED;
    if (cfg->precision != CTU_FP64 && cfg->precision != CTU_MIXED && cfg->precision != CTU_MIXED_IFACE64)
        return CTU_EINVAL;
    if (!(cfg->cfl > 0.0 && cfg->cfl <= 1.0)) return CTU_EINVAL;
    if (!(cfg->glm_alpha >= 0.0)) return CTU_EINVAL;
    if (cfg->nghost != 4) return CTU_EINVAL;
    if (cfg->trace_mode != CTU_TRACE_ALL && cfg->trace_mode != CTU_TRACE_UPWIND) return CTU_EINVAL;
    ctu_ctx *ctx = new (std::nothrow) ctu_ctx();
    if (!ctx) return CTU_ENOMEM;
    ctx->cfg = *cfg;
    if (cudaGetDevice(&ctx->device) != cudaSuccess ||
        cudaMalloc(&ctx->dstatus, sizeof(unsigned int)) != cudaSuccess ||
        cudaMalloc(&ctx->dmax, sizeof(unsigned long long)) != cudaSuccess ||
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
    if (ctx->dwin) cudaFree(ctx->dwin);
    delete ctx->prof;
    delete ctx;
}

__global__ void k_dt_finalize(const unsigned long long *m, double cfl, double dxmin, double *dtch)
{
    const double M = __longlong_as_double((long long)*m);
    const double dt = cfl / M;
    dtch[0] = dt;
    dtch[1] = cfl * dxmin / dt;
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
    if (ctx->cfg.precision != CTU_FP64)
        launch_maxspeed<float>(a, ctx->max_interior, ctx->dmax, s, ctx->prof);
    else
        launch_maxspeed<double>(a, ctx->max_interior, ctx->dmax, s, ctx->prof);
    k_dt_finalize<<<1, 1, 0, s>>>(ctx->dmax, ctx->cfg.cfl, ctx->dxmin, d_dt_ch);
    CTU_CUDA(cudaGetLastError());
    if (h_dt_ch) {
        CTU_CUDA(cudaMemcpyAsync(h_dt_ch, d_dt_ch, 2 * sizeof(double), cudaMemcpyDeviceToHost, s));
        CTU_CUDA(cudaStreamSynchronize(s));
    }
    return CTU_OK;
}

ctu_status ctu_step(ctu_ctx *ctx, const double *U_in, double *U_out, int64_t stride,
                    const ctu_patch *patches, int npatch, const double *d_dt_ch, void *stream)
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
    LaunchInfo li;
    li.max_cells = ctx->max_cells;
    li.recon = ctx->cfg.recon == CTU_PPM;
    li.win = ctx->dwin;
    li.nwin = ctx->reg ? ctx->nwin : 0;
    li.reg = ctx->reg;
    li.scratch = ctx->scratch;
    li.prof = ctx->prof;
    li.iface64 = ctx->cfg.precision == CTU_MIXED_IFACE64;
    if (ctx->cfg.precision != CTU_FP64)
        ctx->last_launches = launch_step<float>(a, li, s);
    else
        ctx->last_launches = launch_step<double>(a, li, s);
    CTU_CUDA(cudaGetLastError());
    return CTU_OK;
}

ctu_status ctu_flux_registers(ctu_ctx *ctx, double *reg, const ctu_flux_window *win, int nwin)
{
    if (!ctx || nwin < 0) return CTU_EINVAL;
    if (!reg || nwin == 0) {
        ctx->reg = nullptr;
        ctx->nwin = 0;
        return CTU_OK;
    }
    if (!win || nwin > 65535) return CTU_EINVAL;
    std::vector<DevWindow> w(nwin);
    for (int i = 0; i < nwin; ++i) {
        const ctu_flux_window &x = win[i];
        if (x.patch < 0 || x.dir < 0 || x.dir >= ctx->cfg.ndim || x.a1 < x.a0 || x.b1 < x.b0 || x.dst < 0)
            return CTU_EINVAL;
        w[i].patch = x.patch; w[i].dir = x.dir; w[i].plane = x.plane;
        w[i].a0 = x.a0; w[i].a1 = x.a1; w[i].b0 = x.b0; w[i].b1 = x.b1; w[i].pad = 0;
        w[i].weight = x.weight; w[i].dst = x.dst;
    }
    CTU_CUDA(cudaDeviceSynchronize());
    if (ctx->dwin) cudaFree(ctx->dwin);
    ctx->dwin = nullptr;
    CTU_CUDA(cudaMalloc(&ctx->dwin, sizeof(DevWindow) * nwin));
    CTU_CUDA(cudaMemcpy(ctx->dwin, w.data(), sizeof(DevWindow) * nwin, cudaMemcpyHostToDevice));
    ctx->nwin = nwin;
    ctx->reg = reg;
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
    long long bx = (ctx->max_cells + 255) / 256;
    if (bx > (1LL << 20)) bx = 1LL << 20;
    k_fill_periodic<<<dim3((unsigned)bx, (unsigned)npatch, 1), 256, 0, s>>>(ctx->dpatch, ctx->cfg.ndim, U, stride);
    CTU_CUDA(cudaGetLastError());
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
