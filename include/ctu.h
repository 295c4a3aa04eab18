/*
 * ctu.h -- C ABI of the GB300 CTU-MHD patch integrator (libctu.so).
 *
 * The library advances batches of ghost-filled patches of an ideal-MHD
 * (GLM-cleaned) state by one dimensionally unsplit Corner Transport Upwind
 * step, following Mignone et al., "The PLUTO code for adaptive mesh
 * computations in astrophysical fluid dynamics" (ApJS 198, 7, 2012):
 *   - equations: Section 2.1, Eq. (1)-(2) (ideal MHD, ideal gas) and
 *     Section 3, Eq. (glm2x2) (GLM divergence cleaning, psi source split);
 *   - time step: Section 3.1, Eq. (Ca);
 *   - step:      Section 3.1, Eq. (update), (incrementop_hyp), (ctu_flux),
 *                (transv) with Pi = 0; Section 3.2 (characteristic
 *                normal predictor, PPM / MC-linear reconstruction);
 *   - flux registers: Section 4.2, Eq. (fluxcorr).
 *
 * Data layout (all arrays are caller-owned device memory unless stated):
 *   A "pool" holds 9 conservative variables in structure-of-arrays form,
 *   U[q * stride + cell], q = 0..8 = (rho, m_x, m_y, m_z, E, B_x, B_y, B_z,
 *   psi), float64.  A patch occupies cells base .. base + NX*NY*NZ - 1 of the
 *   pool, x fastest: cell = base + (k * NY + j) * NX + i, with
 *   N_d = n_d + 2 * 4 for active dimensions (d < ndim) and N_d = n_d = 1 for
 *   inactive ones.  Ghost cells must be filled by the caller before a call.
 *   stride >= base + NX*NY*NZ for every patch; patches must not overlap.
 *
 * Streams: every call that takes `stream` (a cudaStream_t passed as void*)
 * only enqueues work on it, except where "synchronises" is stated.
 *
 * Errors: host-side validation errors are returned at once.  Device-side
 * conditions (a state with rho <= 0 or p <= 0, a NaN, a relativistic
 * recovery that did not converge or gave |v| >= 1) set sticky bits in a
 * device status word that ctu_status_sync() returns and clears.  The library
 * never traps, asserts or exits.
 */
#ifndef CTU_H
#define CTU_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
    CTU_OK = 0,
    CTU_EINVAL = 1,        /* bad argument (null pointer, size, config value) */
    CTU_ENOMEM = 2,        /* device or pinned-host allocation failed */
    CTU_ECUDA = 3,         /* a CUDA runtime call failed */
    CTU_EUNSUPPORTED = 4,  /* valid but not implemented combination */
    CTU_ENEGATIVE = 5,     /* device: a state with rho <= 0 or p <= 0 was met */
    CTU_ENAN = 6,          /* device: a NaN/Inf was met */
    CTU_ERECOVERY = 7,     /* device: primitive recovery did not converge */
    CTU_ESUPERLUMINAL = 8, /* device: |v| >= 1 in relativistic MHD */
    CTU_ETIMEOUT = 9,      /* device: a bounded wait gave up */
    CTU_ETOOLARGE = 10     /* ctu_step_noalloc: batch exceeds its fixed scratch */
} ctu_status;

enum { CTU_MHD = 0, CTU_SRMHD = 1 };
enum { CTU_EOS_IDEAL = 0, CTU_EOS_TM = 1 };
/* reconstruction (Section 3.2) of the characteristic variables:
 *   CTU_LINEAR_MC        linear, Eq. (Linear), MC slope Eq. (MClim)
 *   CTU_PPM              PPM, Eq. (ppm1) + parabolic limiter (ppm_parabolic_lim)
 *   CTU_LINEAR_MINMOD    linear with the MinMod slope, Eq. (minmod)
 *   CTU_LINEAR_HARMONIC  linear with the harmonic-mean slope, Eq. (harmonic_lim)
 *   CTU_LINEAR_VANALBADA linear with the Van Albada slope, Eq. (vanalbada_lim)
 *   CTU_WENO3            improved third-order WENO, Eq. (WENO3), (WENO3a); its
 *                        weights take the characteristic variables of the
 *                        Roe-Balsara normalised left eigenvectors
 * The last four: ideal MHD in CTU_FP64 or CTU_MIXED (CTU_MIXED_IFACE64 and
 * ctu_step_noalloc return CTU_EUNSUPPORTED). */
enum { CTU_LINEAR_MC = 0, CTU_PPM = 1, CTU_LINEAR_MINMOD = 2, CTU_LINEAR_HARMONIC = 3, CTU_LINEAR_VANALBADA = 4,
       CTU_WENO3 = 5 };
enum { CTU_CHAR_TRACE = 0, CTU_MUSCL_HANCOCK = 1 };
/* Riemann solver: CTU_HLLD (MHD; Miyoshi & Kusano 2005), CTU_HLL (SRMHD),
 * CTU_HLLC (MHD; Li 2005: PPM or MC-linear, trace modes ALL or UPWIND,
 * CTU_FP64 or CTU_MIXED, no hybrid integration; else CTU_EUNSUPPORTED).
 * The first-order transverse fluxes take the same solver. */
enum { CTU_HLLD = 0, CTU_HLL = 1, CTU_HLLC = 2 };
/* precision:
 *   CTU_FP64          all arithmetic in float64.
 *   CTU_MIXED         tracing, characteristic projections, Riemann fluxes and
 *                     flux differences in float32; the state and the update
 *                     accumulation in float64.  The cell-centre pressure
 *                     p = (Gamma-1)(E - m^2/2rho - B^2/2) is recovered from
 *                     the float64 state in double-float arithmetic (pairs of
 *                     floats, about 2^-44 relative to E) on the float32
 *                     pipe, not in float64; the n+1/2 interface pressure is
 *                     recovered in an exact increment form that has no
 *                     catastrophic cancellation and so runs in float32.
 *   CTU_MIXED_IFACE64 the literal split: as CTU_MIXED, but every pressure
 *                     recovery runs in plain float64 -- the cell-centre
 *                     states (the step's primitives and both CFL speeds)
 *                     and the interface states, which are formed as float64
 *                     conservative states.  PPM and MC-linear only. */
enum { CTU_FP64 = 0, CTU_MIXED = 1, CTU_MIXED_IFACE64 = 2 };
/* trace_mode: Section 3.2 normal predictor with w_ref = w_(+/-).
 *   CTU_TRACE_ALL    every characteristic field is traced to both
 *                    interfaces (no reference state); second order for
 *                    smooth flows with HLLD, the default.
 *   CTU_TRACE_UPWIND the literal upwind selection beta_+ = [nu > 0],
 *                    beta_- = [nu < 0].
 *   CTU_TRACE_CENTER upwind selection with the reference state w_ref =
 *                    w_(i,0), the cell-centre value.
 *   CTU_TRACE_CW84   upwind selection with Colella & Woodward's reference
 *                    state: the field traced with nu_max = max(0, (u + c_f)
 *                    dt/dx) to the + and nu_min = min(0, (u - c_f) dt/dx) to
 *                    the - interface.
 * The last two: ideal MHD in CTU_FP64 or CTU_MIXED (CTU_MIXED_IFACE64 and
 * ctu_step_noalloc return CTU_EUNSUPPORTED). */
enum { CTU_TRACE_ALL = 0, CTU_TRACE_UPWIND = 1, CTU_TRACE_CENTER = 2, CTU_TRACE_CW84 = 3 };

typedef struct {
    int physics;      /* CTU_MHD: ideal MHD (Section 2.1), requires
                         predictor CTU_CHAR_TRACE and riemann CTU_HLLD.
                         CTU_SRMHD: special-relativistic MHD (Section 2.2),
                         requires predictor CTU_MUSCL_HANCOCK (Section 3.3),
                         riemann CTU_HLL and recon CTU_LINEAR_MC; its
                         primitive recovery (Newton-Raphson) is float64 in
                         both precisions.  Other combinations return
                         CTU_EUNSUPPORTED. */
    int eos;          /* CTU_EOS_IDEAL: ideal gas, Eq. (gammaEos);
                         CTU_EOS_TM: Taub-Mathews, Eq. (TMEos), CTU_SRMHD only
                         (CTU_MHD returns CTU_EUNSUPPORTED) */
    double gamma;     /* ratio of specific heats, > 1 (ignored with CTU_EOS_TM) */
    int ndim;         /* 1, 2 or 3 active dimensions; v_z, B_z always carried */
    int recon;        /* CTU_LINEAR_MC, CTU_PPM, ... (above; Section 3.2) */
    int predictor;    /* CTU_CHAR_TRACE (MHD) or CTU_MUSCL_HANCOCK (SRMHD) */
    int riemann;      /* CTU_HLLD or CTU_HLLC (MHD), CTU_HLL (SRMHD) */
    int precision;    /* CTU_FP64, CTU_MIXED or CTU_MIXED_IFACE64 (above) */
    double cfl;       /* C_a of Eq. (Ca): <= 1 in 2D, <= 1/2 in 3D */
    double glm_alpha; /* c_h^2/c_p^2 = glm_alpha * c_h / min(dx): psi decays by
                         exp(-glm_alpha c_h dt / min dx) per step */
    int nghost;       /* must be 4 */
    int trace_mode;   /* CTU_TRACE_* (above) */
    /* Optional floors of the updated state, >= 0, 0 = off; CTU_MHD only
     * (CTU_SRMHD with a floor returns CTU_EUNSUPPORTED).  The paper fixes no
     * floor: its safeguard against non-physical states is the shock-flagged
     * hybrid integration of its appendix on shock detection (shock_detect
     * below).
     * After the update and the psi damping of every ctu_step, an interior
     * cell with rho < rho_floor takes rho = rho_floor (m, E, B, psi kept);
     * then, with that density, a cell with
     * p = (Gamma-1)(E - m^2/(2 rho) - B^2/2) < p_floor takes
     * E = p_floor/(Gamma-1) + m^2/(2 rho) + B^2/2, in float64 in every
     * precision.  Floored cells are counted (ctu_floor_count).  A
     * non-positive state met inside a step (cell centres, interface states)
     * still sets CTU_ENEGATIVE with floors on. */
    double p_floor;
    double rho_floor;
    /* The hybrid integration of the paper's appendix on shock detection
     * (shock_detect = 1; 0 = off): a cell within three layers of the
     * interior is shocked when
     *   sum_d |q(c + e_d) - q(c - e_d)| / min(q(c + e_d), q(c - e_d))
     *   > shock_eps  and  div v < 0 (central differences),
     * q the thermal (shock_q = 0) or magnetic (1, B^2/2) pressure of the
     * step's initial state.  The faces of shocked cells take the HLL solver
     * (first-order and n+1/2 fluxes) and cells whose reconstruction stencil
     * reaches a shocked cell take linear MinMod reconstruction.  The paper's
     * default threshold is 5.  Ideal MHD with CTU_PPM or CTU_LINEAR_MC,
     * trace_mode CTU_TRACE_ALL or CTU_TRACE_UPWIND, CTU_FP64 or CTU_MIXED
     * (else CTU_EUNSUPPORTED); not in ctu_step_noalloc. */
    int shock_detect;
    int shock_q;
    double shock_eps;
    /* Thermal conduction, the parabolic term of Section 3.1 (Pi != 0):
     * kappa >= 0 the isotropic conductivity of the classical heat flux
     * (Eq. tc_flux with q -> infinity and kappa_par = kappa_perp = kappa),
     * Pi_E = kappa grad T with T = p / rho; 0 = off.  Face fluxes are the
     * central differences Pi_(d,+) = kappa (T(c + e_d) - T(c)) / dx_d, and
     * L_P = sum_d (Pi_(d,+) - Pi_(d,-)) / dx_d (energy only) enters
     *   - every direction's predictor at t^n (Eq. transv), from U^n, and
     *   - the update (Eq. update) at n+1/2, from the cell-centred
     *     U^(n+1/2) = U^n + dt/2 (sum_d L_(H,d)^n + L_P^n), L_(H,d)^n the
     *     first-order Godunov divergences.
     * The CFL rate of ctu_dt and ctu_step_next_dt gains
     * sum_d 2 D / dx_d^2, D = (Gamma-1) kappa / rho (Eq. Ca).  Ideal MHD with
     * CTU_PPM or CTU_LINEAR_MC, CTU_HLLD, trace_mode CTU_TRACE_ALL or
     * CTU_TRACE_UPWIND, no hybrid integration, CTU_FP64 or CTU_MIXED (else
     * CTU_EUNSUPPORTED).  T^(n+1/2) and the update's parabolic term are
     * float64 (CTU_FP64) or double-float with a float64 energy update
     * (CTU_MIXED).  Bound flux registers take the energy flux
     * F_E - Pi_E^(n+1/2) through their faces.  Not in ctu_step_noalloc. */
    double kappa;
    /* Viscosity, the other parabolic term built: nu >= 0 the constant
     * kinematic viscosity of the stress of Eq. (visc_tens),
     * tau = rho nu (grad v + grad v^T - (2/3) I div v); 0 = off.  Momentum flux
     * tau and energy flux v . tau per face, with the normal derivative as for
     * kappa, each transverse derivative the mean of the two cells' central
     * differences, rho and v at the face those of the mean conserved state.
     * It enters the predictors, the update and the registers as kappa does,
     * and the CFL diffusion coefficient becomes
     * D = max((Gamma-1) kappa / rho, (4/3) nu).  Same combinations as kappa. */
    double nu;
    /* Resistivity, the third parabolic term: eta >= 0 constant, the
     * induction term -curl(eta J), J = curl B, i.e. the flux of B_i along d is
     * eta (dB_i/dx_d - dB_d/dx_i), with the energy flux -eta J x B (B_f . that
     * flux, B_f the mean of the two cells); 0 = off.  Derivatives as for nu;
     * it enters the predictors, the update and the registers as kappa does,
     * and D = max((Gamma-1) kappa / rho, (4/3) nu, eta).  Same combinations as
     * kappa. */
    double eta;
    /* Anisotropic conduction: kappa_par >= 0 the conductivity along the
     * field, kappa then being the one across it (Eq. tc_flux, classical):
     * Pi_E = kappa grad T + (kappa_par - kappa) b (b . grad T), b = B_f / |B_f|
     * the direction of the face's mean field (isotropic where B_f = 0), the
     * transverse derivatives of T as for nu.  0 = equal to kappa (isotropic).
     * The CFL diffusion coefficient takes max(kappa, kappa_par).  Same
     * combinations as kappa. */
    double kappa_par;
    /* Saturated conduction (the paper's appendix on the heat flux): tc_phi > 0
     * the parameter phi of the saturated flux q = 5 phi rho c_iso^3.  Each face
     * carries q F_d / (|F| + q), F the classical flux above (its full face
     * gradient of T), q = 5 phi p_u^(3/2) / sqrt(rho_f) with p_u the pressure of
     * the upwind cell (the left one when F_d < 0) and rho_f the mean density.
     * 0 = classical.  The CFL rate keeps the classical coefficients. */
    double tc_phi;
    /* Corner coupling of the transverse terms, Section 3.1:
     *   CTU_CORNER_CELL  the first-order Godunov fluxes between cell-centred
     *                    states of Eq. (transv), the form the paper gives
     *                    for Pi != 0 (default);
     *   CTU_CORNER_MT    the case Pi = 0 "as illustrated by MT" (Mignone &
     *                    Tzeferacos 2010): the transverse fluxes from Riemann
     *                    problems between the normal predictor states of the
     *                    other directions, F*_d = R(U*_(c,+), U*_(c+e_d,-)).
     *                    Six Riemann problems per zone as well; ideal MHD,
     *                    PPM or MC-linear, HLLD, trace modes ALL or UPWIND,
     *                    no hybrid integration and no parabolic terms,
     *                    CTU_FP64 or CTU_MIXED; else CTU_EUNSUPPORTED. */
    int corner;
} ctu_config;
enum { CTU_CORNER_CELL = 0, CTU_CORNER_MT = 1 };

typedef struct {
    int32_t n[3];     /* interior cells per dimension (1 for inactive ones) */
    double dx[3];     /* cell widths; face areas and volumes are Cartesian */
    int64_t base;     /* pool offset of the first (ghost) cell */
    int32_t level;    /* AMR level, informational */
    int32_t flags;    /* reserved, 0 */
} ctu_patch;

/* A flux-register window, Eq. (fluxcorr): faces normal to `dir` on plane
 * `plane` of patch `patch` (0 <= plane <= n_dir; plane p separates interior
 * cells p-1 and p), transverse ranges a in [a0, a1), b in [b0, b1) where
 * (a, b) are the two other dimensions in increasing order.  During every
 * ctu_step that advances this patch, for each such face and variable q:
 *   reg[dst + (q * nb + (b - b0)) * na + (a - a0)] += weight * dt * A * F_q
 * with na = a1 - a0, nb = b1 - b0, A the face area (product of the two
 * transverse cell widths) and F the time-centred flux through the face in
 * the +dir direction. */
typedef struct {
    int32_t patch;    /* index into the ctu_patch array of the ctu_step call */
    int32_t dir;      /* 0, 1, 2 */
    int32_t plane;
    int32_t a0, a1, b0, b1;
    int32_t pad;
    double weight;
    int64_t dst;      /* offset in doubles into the bound register array */
} ctu_flux_window;

typedef struct ctu_ctx ctu_ctx;

/* Validate `cfg`, create a context on the current CUDA device.  *out is
 * library-owned; release it with ctu_destroy. */
ctu_status ctu_init(const ctu_config *cfg, ctu_ctx **out);

/* CFL time step, Eq. (Ca): M = max over the interior cells of all patches of
 * max_d (|v_d| + c_f,d) / dx_d (+ sum_d 2 D / dx_d^2 with the parabolic
 * terms, D = max((Gamma-1) max(kappa, kappa_par) / rho, (4/3) nu, eta)); then
 * dt = cfl / M and
 * c_h = M * min dx (the GLM speed, equal to cfl * min dx / dt).  Writes {dt, c_h} to the device
 * array d_dt_ch[2]; if h_dt_ch is non-null it also copies them there and
 * synchronises the stream.  U: device pool; patches: host array. */
ctu_status ctu_dt(ctu_ctx *ctx, const double *U, int64_t stride,
                  const ctu_patch *patches, int npatch,
                  double *d_dt_ch, double *h_dt_ch, void *stream);

/* One CTU step of every patch: interior cells of U_out receive U_in advanced
 * by dt, with {dt, c_h} read from the device array d_dt_ch[2].  Ghost cells
 * of U_out are not written.  U_in and U_out must not alias.  Bound flux
 * windows whose patch index is < npatch accumulate into the bound register
 * array.  The first call with a new patch list uploads the list and may
 * allocate scratch; make that call before any stream capture. */
ctu_status ctu_step(ctu_ctx *ctx, const double *U_in, double *U_out, int64_t stride,
                    const ctu_patch *patches, int npatch, const double *d_dt_ch,
                    void *stream);

/* ctu_step, and in the same pass the CFL time step of the result: writes
 * {dt, c_h} of U_out's interior cells (as ctu_dt would compute them, in the
 * context's precision) to the device array d_dt_ch_next[2], which must not
 * alias d_dt_ch.  This is the step's fused epilogue of Eq. (Ca), so a time
 * loop needs ctu_dt only before its first step. */
ctu_status ctu_step_next_dt(ctu_ctx *ctx, const double *U_in, double *U_out, int64_t stride,
                            const ctu_patch *patches, int npatch, const double *d_dt_ch,
                            double *d_dt_ch_next, void *stream);

/* The number of interior cells the floors (ctu_config.p_floor, rho_floor)
 * changed since the context was created or this function last returned;
 * resets the count.  Synchronises the stream.  *count is a host int64. */
ctu_status ctu_floor_count(ctu_ctx *ctx, int64_t *count, void *stream);

/* ---- Same-level ghost exchange (Section 4, level advance) ---------------
 * A patch's ghost cells that lie over the interior of a sibling patch (or a
 * periodic image of one) take the sibling's values; a box lists such cells.
 * Box b covers the destination cells x in [lo, hi) -- interior coordinates
 * of the destination patch, ghosts included (-4 .. n+3 on active
 * dimensions; 0 .. 1 on inactive ones) -- and reads source cell x + shift
 * of the source patch (within its ghosted extent).  All nine variables are
 * copied. */
typedef struct {
    int32_t dn[3];    /* destination patch interior extent */
    int32_t sn[3];    /* source patch interior extent */
    int32_t lo[3];    /* destination cells [lo, hi) */
    int32_t hi[3];
    int32_t shift[3]; /* source cell = destination cell + shift */
    int32_t pad;
    int64_t dbase;    /* pool offset of the destination patch's first ghost cell */
    int64_t sbase;    /* pool offset of the source patch's first ghost cell */
} ctu_copy_box;

/* Copy every box from U_src into U_dst (pools of stride sstride / dstride;
 * they may be the same pool, but no cell a box writes may be read by any
 * box of the same call).  Errors: CTU_EINVAL when a box leaves its patch's
 * ghosted extent or a patch leaves its pool.  Enqueues on `stream`; the
 * first call with a new box list uploads it (synchronises). */
ctu_status ctu_copy(ctu_ctx *ctx, double *U_dst, int64_t dstride, const double *U_src, int64_t sstride,
                    const ctu_copy_box *boxes, int nbox, void *stream);

/* For an exchange between processes: ctu_pack writes the source cells of
 * every box, box after box, each as float64 [q][z][y][x] over the box's
 * extent, into the device buffer buf (9 * sum of box cells doubles);
 * ctu_unpack writes such a buffer into the destination cells.  Only the
 * source (pack) or destination (unpack) fields of a box are used. */
ctu_status ctu_pack(ctu_ctx *ctx, double *buf, const double *U_src, int64_t sstride,
                    const ctu_copy_box *boxes, int nbox, void *stream);
ctu_status ctu_unpack(ctu_ctx *ctx, double *U_dst, int64_t dstride, const double *buf,
                      const ctu_copy_box *boxes, int nbox, void *stream);

/* ---- Refinement tagging (Section 4, refinement criteria) ----------------
 * The quantity sigma(U) the criterion is taken of: density (rho, or D in
 * relativistic MHD), total energy density E, B^2/rho, E/rho. */
enum { CTU_TAG_DENSITY = 0, CTU_TAG_ENERGY = 1, CTU_TAG_B2_OVER_RHO = 2, CTU_TAG_E_OVER_RHO = 3 };

/* Eq. (RefCrit), the second-derivative error norm: for every interior cell
 * of every patch,
 *   chi = sqrt( sum_d (D+ - D-)^2 / sum_d (|D+| + |D-| + eps sigma_ref,d)^2 )
 * over the active dimensions d, with D+ = sigma(c + e_d) - sigma(c),
 * D- = sigma(c) - sigma(c - e_d) and sigma_ref,d = |sigma(c + e_d)| +
 * 2 |sigma(c)| + |sigma(c - e_d)|; the cell is tagged when chi > chi_r.  A
 * cell whose denominator is 0 has chi = NaN and no tag.  Every decision is
 * the one float64 evaluation of the definition, in the order written, would
 * take (cells that a float32 evaluation cannot decide with certainty are
 * re-evaluated in float64).
 *   U, stride, patches, npatch: as for ctu_step (one ghost layer is read).
 *   sigma: CTU_TAG_*;  eps >= 0 (the paper uses 0.01);  chi_r >= 0.
 *   tags: device uint8 array in the pool layout (>= stride entries):
 *         tags[base + ghosted cell] = 1 or 0 for every interior cell; other
 *         entries are not written.
 *   d_count: nullable device int64 array of npatch entries: set to the
 *         number of tagged cells of each patch.
 *   chi: nullable device float64 array in the pool layout: when given,
 *         every interior cell's chi is written (and every cell is evaluated
 *         in float64).
 * Enqueues on `stream`; the first call with a new patch list uploads its
 * table (synchronises).  Errors: CTU_EINVAL for a bad argument or patch. */
ctu_status ctu_tag(ctu_ctx *ctx, const double *U, int64_t stride, const ctu_patch *patches, int npatch,
                   int sigma, double eps, double chi_r, unsigned char *tags, int64_t *d_count,
                   double *chi, void *stream);

/* Bind (or, with reg == NULL or nwin == 0, unbind) flux-register windows.
 * `win` is a host array copied at call time; `reg` is a device float64 array
 * the caller owns and zeroes.  Windows must not overlap in reg. */
ctu_status ctu_flux_registers(ctu_ctx *ctx, double *reg, const ctu_flux_window *win,
                              int nwin);

/* Tile autotuner (launch configuration only; the paper has no counterpart).
 * A launch covers every patch shape of the batch; per shape, the kernels use
 * a thread-tile width along x (8, 16 or 32 lanes) and a marching segment
 * length along y and z (4 to 64 cells).  ctu_autotune times ctu_step on the
 * caller's batch for each candidate pair of every shape in turn (largest
 * shapes first, the others held fixed), keeps the fastest, and stores the
 * choice per shape in the context for every later call.  The choice changes
 * only how cells map to threads: each cell's arithmetic, and so the result,
 * is the same for every choice.  U_out is overwritten (U_in is read only);
 * the bound flux registers are left untouched; d_dt_ch is read as in
 * ctu_step.  Synchronises the stream; make the call before any capture.
 * Errors: as ctu_step. */
ctu_status ctu_autotune(ctu_ctx *ctx, const double *U_in, double *U_out, int64_t stride,
                        const ctu_patch *patches, int npatch, const double *d_dt_ch,
                        void *stream);

/* The tile width *xw and segment length *seg the context uses for patches of
 * interior shape n[3] (autotuned if ctu_autotune saw that shape, else the
 * default rule: 32 lanes for n[0] >= 24, 16 for n[0] >= 12, else 8; 16
 * cells). */
ctu_status ctu_tile_params(ctu_ctx *ctx, const int n[3], int *xw, int *seg);

/* ---- Level operators (Section 4 of Mignone et al. 2012; Cartesian) ------
 * The data-parallel operators that produce ctu_step's inputs on a finer
 * level and consume its flux registers: prolongation of a coarse level into
 * fine cells (ghost zones, or new patches), with the coarse solution
 * interpolated in time between two coarse states (Eq. prolong, Eq. intalpha);
 * restriction of a fine level onto the coarse cells it covers (Eq. avgdown);
 * and the flux correction of coarse cells beside coarse-fine interfaces
 * from the flux registers (Eq. fluxcorr, Eq. addreflux).  All arrays are the
 * callers' float64 pools (same layout as ctu_step: [q * stride + cell], 4
 * ghost cells per side on active dimensions, x fastest); the descriptor
 * arrays are host arrays, copied to the device on the first call with new
 * contents (that call synchronises the stream: make it before any capture;
 * later calls with identical descriptors enqueue kernels only).  Returns
 * CTU_EINVAL, on the host, for a descriptor that would reach outside a
 * patch's ghosted region, and for a box whose kernel threads reach 2^31
 * (ctu_prolong: 9 per coarse cell under the box; ctu_restrict: one per
 * coarse cell). */
typedef struct {
    int fn[3];        /* interior cells of the fine patch (1 on inactive dimensions) */
    int cn[3];        /* interior cells of the coarse patch */
    int64_t fbase;    /* pool offset of the fine patch's first ghosted cell */
    int64_t cbase;    /* pool offset of the coarse patch's first ghosted cell */
    int lo[3], hi[3]; /* box of cells, interior coordinates (ghosts: -4..-1, n..n+3):
                         fine cells for ctu_prolong, coarse cells for ctu_restrict */
    int origin[3];    /* coarse cell holding the fine patch's cell 0: fine cell x lies in
                         coarse cell origin + floor(x / ratio) on every active dimension */
    int ratio;        /* refinement ratio, 1 to 4 */
    int phys;         /* ctu_prolong: bit 2d (2d + 1) set when the coarse patch's first
                         (last) interior cell along d touches the physical domain boundary;
                         such a cell's slope along d is the one-sided difference to its
                         neighbour inside the domain (0 when it touches both), and no value
                         beyond the boundary is read.  0 for periodic or interior patches;
                         bits above 5 are invalid.  Ignored by ctu_restrict. */
} ctu_level_box;

/* Eq. (prolong) + Eq. (intalpha): every fine cell x of each box takes
 * U* = (1 - alpha) Uc_old + alpha Uc_new of its coarse cell c, plus, along
 * every active dimension d, (((x_d mod r) + 1/2) / r - 1/2) times the
 * monotonised-central (Eq. MClim) central difference of U* at c, or, for a
 * cell touching the domain boundary (the box's phys bits), the one-sided
 * difference (Section 4).  The coarse cell and its neighbours along each
 * active dimension must lie in the coarse patch's ghosted region.  Uc_old
 * and Uc_new may be the same array. */
ctu_status ctu_prolong(ctu_ctx *ctx, const double *Uc_old, const double *Uc_new, int64_t cstride,
                       double alpha, double *Uf, int64_t fstride, const ctu_level_box *boxes,
                       int nbox, void *stream);

/* Eq. (avgdown): every coarse cell c of each box becomes the mean of its
 * ratio^ndim fine cells (c - origin) * ratio + k, 0 <= k < ratio. */
ctu_status ctu_restrict(ctu_ctx *ctx, double *Uc, int64_t cstride, const double *Uf,
                        int64_t fstride, const ctu_level_box *boxes, int nbox, void *stream);

typedef struct {
    int cn[3];            /* interior cells of the coarse patch */
    int dir, plane, side; /* interface: plane `plane` normal to `dir`; side +1: the corrected
                             coarse cell is `plane` (the interface is its lower face); side -1:
                             the cell is plane - 1 (its upper face) */
    int64_t cbase;        /* pool offset of the coarse patch's first ghosted cell */
    double dx[3];         /* coarse cell widths (the cell volume is their product) */
    int a0, a1, b0, b1;   /* coarse faces [a0, a1) x [b0, b1) in the two other dimensions,
                             increasing order */
    int64_t creg;         /* coarse window in reg, [q][b - b0][a - a0], bound with weight -1 */
    int64_t freg;         /* fine window in reg, [q][fb][fa] of fna x fnb faces, weight +1 */
    int fa0, fb0;         /* fine face of the set's first coarse face */
    int fna, fnb;         /* extents of the fine window */
    int ratio, pad;       /* refinement ratio; pad = 0 */
} ctu_reflux_set;

/* Eq. (fluxcorr) + Eq. (addreflux): after the steps of both levels, each
 * coarse face of each set totals its coarse register sum and the sums of its
 * ratio^(ndim-1) fine faces, and the coarse cell beside it gains side x
 * total / volume.  With the registers bound as stated (coarse -1, fine +1)
 * the total is dt (the space-time average fine flux minus the coarse flux)
 * times the face area.  A cell beside several interfaces gets every
 * correction, in a fixed order: the sets run by class, direction 0..ndim-1
 * and within it side -1 then +1 (one launch each), so the result is
 * reproducible bit for bit and does not depend on the order of `sets`.  The
 * sets of one class reach disjoint cells when the fine patches are disjoint;
 * sets that do share a cell within a class still all land (atomic float64
 * adds), in an order that is then not fixed.  CTU_EINVAL for a set whose
 * 9 x faces reach 2^31. */
ctu_status ctu_reflux(ctu_ctx *ctx, double *Uc, int64_t cstride, const double *reg,
                      const ctu_reflux_set *sets, int nset, void *stream);

/* Conservation diagnostics (a helper, not part of the step): writes to the
 * device array d_out[10] the totals sum over interior cells of U_q times the
 * cell volume (q = 0..8: mass, momentum, energy, magnetic flux, psi) and, in
 * d_out[9], the largest |div B| over interior cells with central
 * differences, sum_d (B_d(c + e_d) - B_d(c - e_d)) / (2 dx_d).  The sums are
 * accumulated with float64 atomics, so their rounding order is not fixed. */
ctu_status ctu_diagnostics(ctu_ctx *ctx, const double *U, int64_t stride,
                           const ctu_patch *patches, int npatch, double *d_out, void *stream);

/* Fill the ghost cells of every patch with periodic copies of its own
 * interior (helper for periodic boxes; not part of the step). */
ctu_status ctu_fill_periodic(ctu_ctx *ctx, double *U, int64_t stride,
                             const ctu_patch *patches, int npatch, void *stream);

/* Synchronise the stream and return (and clear) the sticky device status:
 * CTU_OK or the first device error met since the last call. */
ctu_status ctu_status_sync(ctu_ctx *ctx, void *stream);

/* Static description of a status code. */
const char *ctu_strerror(ctu_status s);

/* Release a context (synchronises the device). */
void ctu_destroy(ctu_ctx *ctx);

/* Number of kernel launches the last ctu_step enqueued (for accounting). */
int ctu_last_launch_count(const ctu_ctx *ctx);

/* Per-kernel timing (measurement aid, not part of the method).  With
 * enable != 0 every kernel the context launches is bracketed by two CUDA
 * events recorded on its stream; totals restart at zero.  enable == 0 turns
 * it off.  Synchronises the device. */
ctu_status ctu_profile(ctu_ctx *ctx, int enable);

/* Synchronises the device, folds the recorded event pairs into per-kernel
 * totals and returns the number of distinct kernel names; if 0 <= i < that
 * number, writes the i-th name (library-owned string), its total device
 * time in ms and its launch count.  Returns 0 when profiling is off. */
int ctu_profile_read(ctu_ctx *ctx, int i, const char **name, double *total_ms, long long *launches);

/* ---- Allocation-free step ------------------------------------------------
 * The paper has no counterpart to this entry point; it serves callers that
 * cannot allocate device memory, such as a host framework whose caching
 * allocator owns all device memory, a real-time loop that cannot take
 * cudaMalloc's implicit synchronisation, or a plug-in that only receives
 * pre-allocated buffers.  ctu_step_noalloc advances the batch exactly as
 * ctu_step does (same kernels, same arithmetic), without flux registers and
 * without a context: its scratch, status word and patch table live in one
 * fixed device array inside libctu.so of CTU_NOALLOC_SCRATCH_BYTES (+ a few
 * KB), held on every GPU that loads the library until the process exits.
 *
 * Limits: npatch <= CTU_NOALLOC_MAX_PATCHES and the scratch the batch needs
 * -- 45 words per ghosted cell (each patch rounded up to 32 cells), 8 bytes
 * for CTU_FP64, 4 for the mixed modes -- must fit in
 * CTU_NOALLOC_SCRATCH_BYTES (one 40^3 patch in FP64, one 56^3 patch mixed);
 * otherwise the call returns CTU_ETOOLARGE and launches nothing.
 *
 * The call allocates nothing (no cudaMalloc/cudaFree, no heap).  Its first
 * call on a device looks up the array's device address (set-up).  The patch
 * table reaches the array in kernel parameters, so no enqueued copy reads
 * host memory after the call returns.  All calls share the one array
 * and it keeps the last call's contents (the status word is cleared at the
 * start of every call): calls that overlap on the GPU -- on different
 * streams, or from different threads -- race and corrupt each other.
 *
 * cfg: as for ctu_init, without floors (a non-zero p_floor or rho_floor
 * returns CTU_EUNSUPPORTED).  U_in, U_out, stride, patches, npatch, d_dt_ch:
 * as for ctu_step.  wait_status != 0: copy the status word back,
 * synchronise the stream and return the device status of this call (CTU_OK,
 * CTU_ENEGATIVE or CTU_ENAN); wait_status == 0: return after enqueueing. */
#define CTU_NOALLOC_SCRATCH_BYTES (48u * 1024u * 1024u)
#define CTU_NOALLOC_MAX_PATCHES 64
ctu_status ctu_step_noalloc(const ctu_config *cfg, const double *U_in, double *U_out,
                            int64_t stride, const ctu_patch *patches, int npatch,
                            const double *d_dt_ch, int wait_status, void *stream);

#ifdef __cplusplus
}
#endif

#endif /* CTU_H */
