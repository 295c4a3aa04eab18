// ctu_noalloc.cu -- ctu_step_noalloc: the CTU step for callers that cannot
// allocate device memory.
//
// ctu_step keeps its intermediate arrays (primitive states, first-order and
// time-centred fluxes, interface states) in scratch that its context obtains
// with cudaMalloc.  Some callers cannot do that: a host framework whose
// caching allocator owns all device memory and forbids allocations behind
// its back, a real-time loop that cannot afford cudaMalloc's implicit device
// synchronisation, or a plug-in that is handed pre-allocated buffers only.
// This entry point runs the same kernels with their scratch, the status word
// and the patch table carved out of one fixed array that lives in this
// module's device image, so the call itself allocates nothing.
//
// Limits: at most CTU_NOALLOC_MAX_PATCHES patches and CTU_NOALLOC_SCRATCH_BYTES
// of scratch (the sum over patches of the ghosted cell count, each rounded
// up to 32 cells, times 45 words of 8 bytes for CTU_FP64 or 4 bytes for the
// mixed modes: one 40^3 patch in FP64, or one 56^3 patch in mixed precision).
// The array occupies CTU_NOALLOC_SCRATCH_BYTES (plus a few KB) on every GPU
// that loads the library, until the process exits.
#include <cuda_runtime.h>

#include <cstring>
#include <mutex>

#include "ctu.h"
#include "ctu_launch.h"

using namespace ctu;

namespace {

constexpr size_t kHeadBytes = 256;  // status word at 0, per-step parameters at 64
constexpr size_t kTableBytes = (sizeof(DevPatch) * CTU_NOALLOC_MAX_PATCHES + 255) / 256 * 256;
constexpr size_t kScratchBytes = (size_t)CTU_NOALLOC_SCRATCH_BYTES;
constexpr size_t kTotalBytes = kHeadBytes + kTableBytes + kScratchBytes;
constexpr int kMaxDevices = 64;

std::mutex g_mu;
unsigned char *g_base[kMaxDevices];  // device address of g_noalloc, per device

} // namespace

// The one device array behind ctu_step_noalloc: [status | patch table | scratch].
static __device__ __align__(256) unsigned char g_noalloc[kTotalBytes];

// Patch descriptors travel to the array by value, in the parameters of a
// small kernel (kChunk per launch, well inside the parameter space), so that
// no copy reads the caller's host stack after the call has returned.
constexpr int kChunk = 16;
struct TableChunk {
    DevPatch p[kChunk];
};
static __global__ void k_put_table(TableChunk c, int n, DevPatch *dst)
{
    const int i = (int)threadIdx.x;
    if (i < n) dst[i] = c.p[i];
}

// Set-up, once per device with that device current: host code cannot use the
// symbol g_noalloc as a device address (on the host it names a stand-in), so
// the real address is looked up and cached.
static ctu_status noalloc_base(unsigned char **out)
{
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) return CTU_ECUDA;
    std::lock_guard<std::mutex> lock(g_mu);
    if (!g_base[dev]) {
        void *p = nullptr;
        const cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc);
        if (e != cudaSuccess || !p) return CTU_ECUDA;
        g_base[dev] = (unsigned char *)p;
    }
    *out = g_base[dev];
    return CTU_OK;
}

extern "C" ctu_status ctu_step_noalloc(const ctu_config *cfg, const double *U_in, double *U_out,
                                       int64_t stride, const ctu_patch *patches, int npatch,
                                       const double *d_dt_ch, int wait_status, void *stream)
{
    if (!cfg || !U_in || !U_out || !d_dt_ch || U_in == U_out || !patches) return CTU_EINVAL;
    if (cfg->physics != CTU_MHD || cfg->eos != CTU_EOS_IDEAL || cfg->predictor != CTU_CHAR_TRACE ||
        cfg->riemann != CTU_HLLD || cfg->p_floor != 0.0 || cfg->rho_floor != 0.0 ||
        (cfg->recon > CTU_PPM && cfg->recon <= CTU_WENO3) ||
        (cfg->trace_mode > CTU_TRACE_UPWIND && cfg->trace_mode <= CTU_TRACE_CW84) || cfg->shock_detect != 0 ||
        cfg->kappa != 0.0 || cfg->kappa_par != 0.0 || cfg->nu != 0.0 || cfg->eta != 0.0 || cfg->tc_phi != 0.0 ||
        cfg->corner != CTU_CORNER_CELL)
        return CTU_EUNSUPPORTED;
    if (!(cfg->gamma > 1.0) || cfg->ndim < 1 || cfg->ndim > 3 || cfg->nghost != 4 ||
        (cfg->recon != CTU_LINEAR_MC && cfg->recon != CTU_PPM) ||
        (cfg->precision != CTU_FP64 && cfg->precision != CTU_MIXED && cfg->precision != CTU_MIXED_IFACE64) ||
        !(cfg->glm_alpha >= 0.0) ||
        (cfg->trace_mode != CTU_TRACE_ALL && cfg->trace_mode != CTU_TRACE_UPWIND))
        return CTU_EINVAL;
    if (npatch <= 0) return CTU_EINVAL;
    if (npatch > CTU_NOALLOC_MAX_PATCHES) return CTU_ETOOLARGE;

    // Patch table and launch groups on the stack (no heap use), and the
    // scratch they need.  Each patch is its own launch group.
    DevPatch table[CTU_NOALLOC_MAX_PATCHES];
    Group groups[CTU_NOALLOC_MAX_PATCHES];
    long long off = 0;
    for (int i = 0; i < npatch; ++i) {
        DevPatch &q = table[i];
        long long cells = 1;
        q.hmin = 1e300;
        for (int d = 0; d < 3; ++d) {
            const int g = d < cfg->ndim ? 4 : 0;
            if (patches[i].n[d] < 1 || patches[i].n[d] > 4096 || (d >= cfg->ndim && patches[i].n[d] != 1) ||
                !(patches[i].dx[d] > 0.0))
                return CTU_EINVAL;
            q.n[d] = patches[i].n[d];
            q.g[d] = g;
            q.N[d] = q.n[d] + 2 * g;
            q.dx[d] = patches[i].dx[d];
            q.idx[d] = 1.0 / q.dx[d];
            q.idxf[d] = (float)q.idx[d];
            if (d < cfg->ndim && q.dx[d] < q.hmin) q.hmin = q.dx[d];
            cells *= q.N[d];
        }
        if (patches[i].base < 0 || patches[i].base + cells > stride) return CTU_EINVAL;
        q.base = patches[i].base;
        q.soff = off;
        off += (cells + 31) / 32 * 32;
        groups[i].first = i;
        groups[i].count = 1;
        for (int d = 0; d < 3; ++d) {
            groups[i].n[d] = q.n[d];
            groups[i].N[d] = q.N[d];
        }
        groups[i].xw = Tiles::xw(q.n[0]);
        groups[i].seg = SEG;
    }
    const size_t elt = cfg->precision == CTU_FP64 ? sizeof(double) : sizeof(float);
    if ((size_t)off * SCRATCH_ARRAYS * elt > kScratchBytes) return CTU_ETOOLARGE;

    unsigned char *base = nullptr;
    ctu_status st = noalloc_base(&base);
    if (st != CTU_OK) return st;
    cudaStream_t s = (cudaStream_t)stream;
    unsigned int *status = (unsigned int *)base;
    StepParams *sp = (StepParams *)(base + 64);
    DevPatch *dtab = (DevPatch *)(base + kHeadBytes);
    void *scratch = base + kHeadBytes + kTableBytes;

    // The array keeps the previous call's contents: the status word must start
    // at zero; the per-step parameters and every scratch word the kernels read
    // are written earlier in the same call, so they need no clearing.
    if (cudaMemsetAsync(status, 0, sizeof(unsigned int), s) != cudaSuccess) return CTU_ECUDA;
    for (int i0 = 0; i0 < npatch; i0 += kChunk) {
        const int m = npatch - i0 < kChunk ? npatch - i0 : kChunk;
        TableChunk c;
        std::memset(&c, 0, sizeof(c));
        for (int i = 0; i < m; ++i) c.p[i] = table[i0 + i];
        k_put_table<<<1, kChunk, 0, s>>>(c, m, dtab + i0);
    }

    StepArgs a;
    std::memset(&a, 0, sizeof(a));
    a.patches = dtab;
    a.npatch = npatch;
    a.ndim = cfg->ndim;
    a.gam = cfg->gamma;
    a.igm = 1.0 / (cfg->gamma - 1.0);
    a.gamf = (float)cfg->gamma;
    a.gm1f = (float)(cfg->gamma - 1.0);
    a.glm_alpha = cfg->glm_alpha;
    a.upwind = cfg->trace_mode;
    a.limiter = cfg->recon;
    a.flags = nullptr;
    a.shock_eps = 0.0;
    a.shock_q = 0;
    a.kappa = 0.0;
    a.nu = 0.0;
    a.eta = 0.0;
    a.kpar = 0.0;
    a.phi = 0.0;
    a.par_cond = a.par_visc = a.par_res = a.par_aniso = a.par_sat = 0;
    a.lp = nullptr;
    a.th = nullptr;
    a.U = U_in;
    a.Uout = U_out;
    a.ustride = stride;
    a.sstride = off;
    a.dtch = d_dt_ch;
    a.sp = sp;
    a.status = status;
    LaunchInfo li;
    li.groups = groups;
    li.ngroups = npatch;
    li.recon = cfg->recon == CTU_PPM;
    li.iface64 = cfg->precision == CTU_MIXED_IFACE64;
    li.physics = PH_MHD;
    li.scratch = scratch;
    li.sp = sp;
    li.prof = nullptr;
    li.sms = 0;  // launch_rows takes 152
    {
        int dev = 0, sms = 0;
        if (cudaGetDevice(&dev) == cudaSuccess &&
            cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) == cudaSuccess)
            li.sms = sms;
    }
    if (cfg->precision == CTU_FP64)
        launch_step<double>(a, li, s);
    else
        launch_step<float>(a, li, s);
    if (cudaGetLastError() != cudaSuccess) return CTU_ECUDA;
    if (!wait_status) return CTU_OK;
    unsigned int h = 0;
    if (cudaMemcpyAsync(&h, status, sizeof(h), cudaMemcpyDeviceToHost, s) != cudaSuccess) return CTU_ECUDA;
    if (cudaStreamSynchronize(s) != cudaSuccess) return CTU_ECUDA;
    if (h & ST_NAN) return CTU_ENAN;
    if (h & ST_NEG) return CTU_ENEGATIVE;
    return CTU_OK;
}
