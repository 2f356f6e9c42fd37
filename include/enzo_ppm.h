/*
 * enzo_ppm.h -- C ABI of the GB300 (sm_103a) directionally split PPM hydro sweep.
 *
 * The library advances the Euler equations of an ideal gas (paper Sec. 2.1:
 * conserved density, momentum and total energy density; EOS e = p/(gamma-1))
 * on a batch of ghost-zoned grid patches (Sec. 3: rectilinear patches with 3
 * ghost layers each, solved as independent problems with Dirichlet ghost
 * zones) by the direct-Eulerian PPM method of Sec. 4.1 (parabolic
 * reconstruction, monotone limiter, characteristic tracing, two-shock Riemann
 * solver with Newton iteration on p*, Sec. 4.1.2, and the conservative
 * update), one split direction per call, with the hydro CFL rule of Sec. 9.
 *
 * Conventions shared by every entry point:
 *   - All array pointers are DEVICE pointers owned by the caller.  Outside the
 *     hierarchy driver (enzo_hierarchy_*, which owns the device state of a
 *     hierarchy, allocated through the caller's allocator or cudaMalloc) the
 *     library allocates nothing and frees nothing; it keeps no state between
 *     calls except a per-device cache of launch sizes and the fixed scratch
 *     array of enzo_ppm_sweep_noalloc.
 *   - Every call is asynchronous on the given stream (NULL = legacy default
 *     stream) unless stated otherwise, and returns ENZO_OK or a negative
 *     ENZO_ERR_* code.  No C++ exception crosses the ABI.
 *   - Numerical events (Newton cap hits, HLL fallbacks, floors, NaN) are not
 *     errors: kernels add them to the caller's device counters `status`
 *     (ENZO_STATUS_WORDS unsigned 64-bit words, indexed by ENZO_ST_*).
 *   - Field storage: five float64 arrays U[0..4] = rho, m_x, m_y, m_z, E (E is
 *     the total energy DENSITY).  Patch p occupies, in every array, the
 *     elements [off, off + (nx+2ng)(ny+2ng)(nz+2ng)), x fastest, then y, z.
 */
#ifndef ENZO_PPM_H
#define ENZO_PPM_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define ENZO_ABI_VERSION 1

/* ---- error codes ---- */
#define ENZO_OK 0
#define ENZO_ERR_ARG (-1)        /* NULL pointer, bad enum, bad size, non-finite dt */
#define ENZO_ERR_CUDA (-2)       /* a CUDA runtime call or launch failed */
#define ENZO_ERR_RANGE (-3)      /* a patch descriptor is out of range, or a batch is larger
                                    than a fixed limit of the call */
#define ENZO_ERR_WORKSPACE (-4)  /* workspace missing or smaller than required */
#define ENZO_ERR_UNSUPPORTED (-5)/* option not available in this library */

/* ---- precision modes ---- */
#define ENZO_FP64 0  /* every step in FP64, no FMA contraction (parity path) */
#define ENZO_FP32 1  /* FP32 reconstruction, tracing and Riemann; FP64 conserved
                        accumulation, and FP64 E - KE in high-Mach cells */

/* ---- Newton starting guess for p* ---- */
#define ENZO_GUESS_PLAIN 0  /* acoustic two-shock guess */
#define ENZO_GUESS_MLP 1    /* learned guess (enzo_mlp_*), plain guess as fallback */

/* ---- patch flags ---- */
#define ENZO_PATCH_PERIODIC 1 /* the patch is its own periodic neighbour: sweeps read
                                 ghost positions from the wrapped active cells and
                                 leave stored ghost cells untouched */

/* ---- status counters (indices into the caller's uint64 status array) ---- */
enum {
    ENZO_ST_INTERFACES = 0,   /* Riemann problems solved */
    ENZO_ST_NEWTON_ITERS = 1, /* Newton updates, summed */
    ENZO_ST_NEWTON_NONCONV = 2,/* interfaces whose Newton hit the cap */
    ENZO_ST_HLL_CELLS = 3,    /* cells that went to rho <= 0 and were re-fluxed with HLL */
    ENZO_ST_NEG_AFTER = 4,    /* cells still failing the fallback's test after it */
    ENZO_ST_RHO_FLOOR = 5,    /* cell densities raised to rho_floor */
    ENZO_ST_P_FLOOR = 6,      /* cell pressures raised to p_floor */
    ENZO_ST_NAN = 7,          /* updated cells holding NaN */
    ENZO_ST_BAD_PATCH = 8,    /* descriptors rejected on the device (skipped) */
    ENZO_ST_FP64_EKE = 9,     /* FP32 mode: cells whose E - KE was redone in FP64 */
    ENZO_ST_GUESS_RESTARTS = 10, /* learned guess abandoned for the plain guess */
    ENZO_ST_GUESS_CALLS = 11, /* interfaces given a learned guess (those past the gate) */
    ENZO_ST_TIMEOUT = 12,     /* bounded waits that ran out (tensor-core kernels) */
    ENZO_ST_GE_PRESSURE = 13, /* ENZO_OPT_DUAL: zone loads whose pressure came from the gas energy */
    ENZO_STATUS_WORDS = 16
};

/* One grid patch (Sec. 3).  n: active cells per axis (>= 1); ng: ghost layers
 * stored on each side (must be 3, the PPM stencil's need, Sec. 3); off: element
 * offset of the patch's first stored cell in every field array; dx: cell widths;
 * level: refinement level (informational); flags: ENZO_PATCH_*. */
typedef struct {
    int32_t n[3];
    int32_t ng;
    int64_t off;
    double dx[3];
    int32_t level;
    int32_t flags;
    int64_t freg_all;   /* offset of this patch's all-face flux register in the batch's
                           freg buffer, or -1.  FP64 sweeps store the final flux of every face
                           (FP32 sweeps the increment dt/dx F the cells applied, in FP64)
                           bounding an active cell: for axis d (x, y, z in order) a block
                           of (n_d+1) n_a1 n_a2 x C doubles at
                           ((j2 n_a1 + j1)(n_d+1) + f) C + v, a1 < a2 the other axes, f the
                           face left of active cell f, v = rho, m_normal, m_a1, m_a2, E.
                           C = 5, or 6 when the batch has a gas-energy field (ge): v = 5
                           is then the gas-energy flux (ENZO_OPT_DUAL, whose sweeps alone
                           may write such registers). */
    int64_t freg_bnd;   /* offset of the boundary-face register, or -1: sweeps ADD dt x flux
                           (FP32 sweeps: the applied increment)
                           of the two faces bounding the patch along d, block of 2 n_a1 n_a2
                           x C doubles per axis at ((j2 n_a1 + j1) 2 + side) C + v.  Used by
                           flux correction (Sec. 3.4); the caller zeroes it before a
                           parent step's subcycles. */
} enzo_patch;

/* A batch of patches that share one timestep (a level, Sec. 3 and Sec. 9). */
typedef struct {
    int32_t npatch;               /* number of descriptors (>= 0) */
    int32_t reserved;
    const enzo_patch *patches;    /* DEVICE array [npatch] */
    int64_t field_len;            /* elements in each U[f]; descriptors reaching
                                     past it are rejected (ENZO_ST_BAD_PATCH) */
    double *U[5];                 /* DEVICE fields rho, m_x, m_y, m_z, E */
    void *workspace;              /* DEVICE scratch, >= enzo_workspace_size(npatch) bytes,
                                     16-byte aligned; contents need no initialisation */
    size_t ws_bytes;
    unsigned long long *status;   /* DEVICE counters [ENZO_STATUS_WORDS]; added to */
    void *stream;                 /* cudaStream_t */
    double *freg;                 /* DEVICE flux registers (see enzo_patch.freg_*), or NULL */
    double *ge;                   /* DEVICE gas-energy field rho e (field_len elements, same
                                     layout as U), or NULL: read and updated only by
                                     sweeps with ENZO_OPT_DUAL; carried whenever non-NULL
                                     by the ghost fills and the hierarchy calls (a sixth
                                     field there, and a sixth flux-register component) */
} enzo_patch_batch;

/* Interface flux solvers (Sec. 4.1.2): the two-shock Riemann solver with a
 * Newton iteration on p*, or the HLL / HLLC approximate solvers on the traced
 * states (Davis signal speeds).  The positivity fallback is HLL in every case. */
enum { ENZO_SOLVER_TWOSHOCK = 0, ENZO_SOLVER_HLL = 1, ENZO_SOLVER_HLLC = 2 };

/* Optional dissipation of the reconstruction (Sec. 4.1 names contact
 * steepening, flattening and a diffusive flux as options and defers to CW84):
 * steepening of the density at contacts, flattening of every variable in zones
 * that compress across a strong pressure jump (the zone's own weight: the
 * stencil stays within three ghost zones), and a flux 0.1 max(0, u_L - u_R)
 * (U_L - U_R) at compressive interfaces.
 * ENZO_OPT_DUAL: the dual energy formulation (Sec. 4.1.1): the batch's ge field
 * (the gas energy rho e) is advected with the mass flux, eps = ge / rho
 * reconstructed and traced like a transverse velocity and upwinded by the sign
 * of u*, plus the source -p_j (u_{j+1/2} - u_{j-1/2}) dt/dx with the zone
 * pressure at the start of the sweep and the Riemann interface velocities
 * (faces re-fluxed by the HLL fallback: the HLL mass flux times the upwind zone
 * eps, the mean zone velocity).  A zone takes its pressure from ge where
 * E - KE < 1e-3 E (eta1), decided in FP64 in both precisions; after the update
 * ge is reset to E - KE where that exceeds 0.1 (eta2) times the largest E of the
 * cell and its two neighbours along the sweep.  Needs the two-shock solver and
 * a non-NULL ge (ENZO_ERR_ARG otherwise).  Flux registers then get the
 * gas-energy flux as a sixth component per face; conversely a batch with
 * both ge and flux registers must be swept with this option (ENZO_ERR_ARG
 * otherwise). */
enum { ENZO_OPT_STEEPEN = 1, ENZO_OPT_FLATTEN = 2, ENZO_OPT_DIFFUSE = 4, ENZO_OPT_DUAL = 8 };

/* Method parameters (Sec. 4.1, 4.1.2, 9). */
typedef struct {
    double gamma;       /* ratio of specific heats, > 1 */
    double cfl;         /* kappa_hydro of Sec. 9, in (0, 1] */
    int32_t precision;  /* ENZO_FP64 | ENZO_FP32 */
    int32_t guess;      /* ENZO_GUESS_PLAIN | ENZO_GUESS_MLP */
    double newton_tol;  /* residual tolerance; <= 0 selects 1e-14 (FP64) / 1e-6 (FP32) */
    int32_t newton_max; /* Newton update cap; <= 0 selects 20 (FP64) / 12 (FP32) */
    int32_t fallback;   /* HLL re-flux (Sec. 4.1.2) of both faces of each cell whose update
                           fails: 0 off; 1 (default) rho <= 0, the paper's trigger; 2 rho <= 0
                           or a non-positive internal energy, 2 rho E - |m|^2 <= 0 (the paper
                           names negative densities or energies; its own kernel instantiations,
                           not with ENZO_GUESS_MLP).  Other values: ENZO_ERR_ARG */
    double rho_floor;   /* density floor, > 0 */
    double p_floor;     /* pressure floor, > 0 */
    const void *mlp;    /* DEVICE weight blob from enzo_mlp_pack (ENZO_GUESS_MLP only;
                           the learned guess runs in the FP32 path; FP64 returns
                           ENZO_ERR_UNSUPPORTED) */
    int32_t tile[3];    /* pencils per CTA tile for sweeps along x, y, z: 0 (default,
                           128), 64, 128 or 256; used by the FP32 plain-guess path
                           (the FP64 and learned paths always use 128).  Picked
                           per batch by the autotuner (paper_1307_2265_gb300.tune). */
    int32_t solver;     /* interface flux (Sec. 4.1.2): ENZO_SOLVER_TWOSHOCK (default, 0),
                           ENZO_SOLVER_HLL or ENZO_SOLVER_HLLC; the learned guess needs the
                           two-shock solver (ENZO_ERR_ARG otherwise) */
    double mlp_gate;    /* ENZO_GUESS_MLP: an interface takes the learned guess only when
                           its jump strength max(|pL-pR|/(pL+pR), |uL-uR|/c_m) exceeds this
                           (c_m^2 = gamma (pL+pR)/(rhoL+rhoR)); weaker interfaces keep the
                           plain guess, which is already within a Newton step of the root
                           there.  0 selects 0.03; < 0 takes the learned guess everywhere.
                           A CTA whose interfaces are all below the gate skips the network. */
    int32_t options;    /* ENZO_OPT_* bits (default 0): the optional reconstruction
                           dissipation of Sec. 4.1 / CW84; not with ENZO_GUESS_MLP */
} enzo_params;

/* Bytes of device workspace a batch of npatch patches needs. */
size_t enzo_workspace_size(int32_t npatch);

/* Host-side check of descriptors before they are uploaded: sizes >= 1 and at
 * most 4096 per axis, ng == 3, dx finite and > 0, patches inside field_len.
 * Returns ENZO_OK, ENZO_ERR_ARG (NULL) or ENZO_ERR_RANGE; *bad_index (may be
 * NULL) receives the first offending index or -1. */
int enzo_validate_patches(const enzo_patch *host_patches, int32_t npatch, int64_t field_len,
                          int32_t *bad_index);

/* One split PPM sweep along axis dir (0 = x, 1 = y, 2 = z) with timestep dt
 * (Sec. 4.1: reconstruction, limiter, tracing, two-shock Riemann, fluxes, FP64
 * conservative update U_j += dt/dx (F_{j-1/2} - F_{j+1/2}), HLL fallback).
 * cover_mask: bit a set means the pencils also cover the ghost layers of
 * transverse axis a (the coverage that lets ghosts be filled once per step:
 * first sweep of a step covers both transverse axes, the second the axis not
 * yet swept, the third none).  Periodic patches ignore cover_mask.  Updates
 * active cells along dir in place; reads ghost cells. */
int enzo_ppm_sweep(const enzo_patch_batch *b, int32_t dir, double dt, int32_t cover_mask,
                   const enzo_params *p);

/* As enzo_ppm_sweep, with dt read on the device from dt_dev (one double, e.g.
 * written by enzo_timestep_cfl), so a sequence of calls needs no host sync and
 * can be captured in a CUDA graph. */
int enzo_ppm_sweep_dev(const enzo_patch_batch *b, int32_t dir, const double *dt_dev,
                       int32_t cover_mask, const enzo_params *p);

/* enzo_ppm_sweep that also logs traced interface states for training the
 * learned guess (not in the paper).  Every interface whose hash of (patch,
 * pencil, position) is divisible by log_stride appends its left and right
 * states (rho_L, u_L, p_L, rho_R, u_R, p_R) as float32 to log[slot][6];
 * *log_count (DEVICE uint64, caller-zeroed) counts appended rows, and rows
 * beyond log_cap are dropped (the count still grows). */
int enzo_ppm_sweep_logged(const enzo_patch_batch *b, int32_t dir, double dt, int32_t cover_mask,
                          const enzo_params *p, float *log, unsigned long long *log_count, int64_t log_cap,
                          int32_t log_stride);

/* Allocation-free variant of enzo_ppm_sweep (the paper has no counterpart;
 * this is an interface convenience).  It is meant for callers that cannot
 * allocate device memory for this library, for instance a host code that owns
 * every device buffer through its own pool, or one whose memory budget is
 * fixed once time stepping starts.  It performs the same sweep with the same
 * arguments and checks as enzo_ppm_sweep (b->patches, b->U, b->status,
 * b->stream, b->freg, b->ge, p->tile ...), but ignores b->workspace and
 * b->ws_bytes (they may be NULL / 0).  Its scratch (the tile table and tile
 * counter) lives in a 128 KiB array of device memory owned by the library.
 * Every GPU that loads the library keeps that array until the process exits.
 *   - At most 32000 patches per call; larger batches return ENZO_ERR_RANGE.
 *   - The first call on a device looks up the array's device address and
 *     caches it.  Make that first call before any stream capture, and do not
 *     keep using the library after cudaDeviceReset.
 *   - All calls share the array.  Each call rewrites the tile table and zeroes
 *     the counter before use, so the previous call's contents do not matter,
 *     but calls whose kernels overlap on the GPU (e.g. on two streams) race on
 *     it.
 *   - Nothing is allocated or freed; ENZO_GUESS_MLP returns ENZO_ERR_UNSUPPORTED. */
int enzo_ppm_sweep_noalloc(const enzo_patch_batch *b, int32_t dir, double dt, int32_t cover_mask,
                           const enzo_params *p);

/* Fill every ghost cell of every non-periodic patch from its own periodic image
 * (Sec. 3.1, periodic boundary, edges and corners included).  Periodic patches
 * are left alone (their sweeps wrap). */
int enzo_ghost_fill_periodic(const enzo_patch_batch *b);

/* Active cells of every patch to (enzo_pack_active) or from (enzo_unpack_active)
 * a packed layout without ghost zones, e.g. a staging copy of a level's state in
 * host memory: patch i's active cells, x fastest, then y, then z, occupy
 * packed[f][act_off[i] ...] for the five fields f (DEVICE arrays; act_off:
 * DEVICE int64 [npatch], chosen by the caller, blocks must not overlap).
 * packed_ge: the same for the gas energy (DEVICE, needs b->ge), or NULL to
 * leave it out.  Unpacking writes active cells only; ghost zones are left as
 * they are (a sweep or a ghost fill derives them).  Uses the batch's workspace
 * and stream.  ENZO_ERR_ARG on NULL arrays. */
int enzo_pack_active(const enzo_patch_batch *b, double *const packed[5], double *packed_ge,
                     const int64_t *act_off);
int enzo_unpack_active(const enzo_patch_batch *b, double *const packed[5], double *packed_ge,
                       const int64_t *act_off);

/* External boundary conditions of a grid (Sec. 3.1 lists reflecting, outflow,
 * inflow and periodic; inflow is not provided). */
enum {
    ENZO_BC_PERIODIC = 0, /* ghost layer g copies the active cell g back from the far face */
    ENZO_BC_REFLECT = 1,  /* mirror image about the face, momentum along the axis negated;
                             needs n >= 3 along that axis (smaller patches get the mirror
                             folded back into the patch) */
    ENZO_BC_OUTFLOW = 2   /* zero gradient: the boundary cell is copied outward */
};

/* Ghost fill of every non-periodic patch as a single grid with external
 * boundaries bc[3] (HOST array: condition along x, y, z; Sec. 3.1).  Edges and
 * corners take every condition that applies (as filling x, then y, then z over
 * the full extents).  Patches flagged ENZO_PATCH_PERIODIC are left alone.
 * Returns ENZO_ERR_ARG for a NULL bc or an unknown condition. */
int enzo_ghost_fill_boundary(const enzo_patch_batch *b, const int32_t bc[3]);

/* Level timestep of Sec. 9: dt = cfl / max over active cells of all patches of
 * sum_d (c_s + |v_d|)/dx_d, with c_s = sqrt(gamma p / rho).  The min-reduction
 * runs on the device.  dt_out: DEVICE pointer to one double when
 * dt_out_on_device != 0 (asynchronous, graph-capturable), else a HOST pointer
 * (the call synchronises the stream). */
int enzo_timestep_cfl(const enzo_patch_batch *b, const enzo_params *p, double *dt_out,
                      int32_t dt_out_on_device);

/* One full step (Sec. 3 control loop for one level, hydro only): ghost fill of
 * non-periodic patches, then the three split sweeps in the order of step
 * `step_index` (x,y,z when even, z,y,x when odd) with the once-per-step ghost
 * coverage.  dt_dev: DEVICE pointer to the step's dt (e.g. written by
 * enzo_timestep_cfl), read by the kernels, so a captured graph replays with
 * each step's own dt. */
int enzo_step(const enzo_patch_batch *b, const enzo_params *p, int32_t step_index,
              const double *dt_dev);

/* As enzo_step with the ghost fill of enzo_ghost_fill_boundary(bc) (HOST bc[3]). */
int enzo_step_boundary(const enzo_patch_batch *b, const enzo_params *p, int32_t step_index,
                       const double *dt_dev, const int32_t bc[3]);

/* Riemann problems on their own (Sec. 4.1.2): n independent interfaces given
 * as SoA DEVICE arrays of left/right primitive states.  Outputs (DEVICE,
 * length n, each may be NULL): pstar, ustar, and the state sampled at x/t = 0
 * (rho_face, u_face, p_face); iters gets the Newton update count, negated when
 * the cap was hit.  pguess (may be NULL): per-interface starting guesses
 * (values <= 0 select the plain guess).  Arrays are float64 when
 * p->precision == ENZO_FP64 and float32 when ENZO_FP32. */
typedef struct {
    int64_t n;
    const void *rhoL, *uL, *pL, *rhoR, *uR, *pR;
    const void *pguess;
    void *pstar, *ustar, *rho_face, *u_face, *p_face;
    int32_t *iters;
    void *stream;
} enzo_riemann_states;

int enzo_riemann_solve(const enzo_riemann_states *s, const enzo_params *p);

/* ---- learned Newton starting guess for p* (not in the paper) ----
 * The two-shock solver of Sec. 4.1.2 iterates on p*.  An MLP 6 -> 64 -> 64 -> 1
 * with SiLU, BF16 weights and FP32 accumulation (tcgen05 tensor cores)
 * predicts y = ln(p* / sqrt(p_L p_R)) from the Riemann-invariant features
 *   (ln rho_L/rho_ref, (u_L-u_bar)/c_ref, ln p_L/p_ref, same for R),
 *   rho_ref = sqrt(rho_L rho_R), p_ref = sqrt(p_L p_R), c_ref = sqrt(gamma p_ref/rho_ref),
 *   u_bar = (u_L+u_R)/2.
 * Newton then starts from p_ref exp(y); if it does not converge it restarts
 * from the plain guess, so answers stay the plain solver's to tolerance.
 * Master parameters: ENZO_MLP_PARAMS float32 values W1[64][6], b1[64],
 * W2[64][64], b2[64], w3[64], b3.  The device blob (ENZO_MLP_BLOB_BYTES,
 * 16-byte aligned) holds the BF16 tensor-core tiles and FP32 vectors the
 * kernels read; enzo_params.mlp points to it. */
#define ENZO_MLP_PARAMS 4673
#define ENZO_MLP_BLOB_BYTES 19456

/* Convert FP32 master parameters (DEVICE) into the blob (DEVICE). */
int enzo_mlp_pack(const float *master, void *blob, void *stream);

/* y[i] = MLP(x[i][0..5]) for n samples (DEVICE, float32).  status: DEVICE
 * counters; ENZO_ST_TIMEOUT counts tensor-core waits that ran out (then the
 * outputs of that CTA are not written). */
int enzo_mlp_forward(const void *blob, const float *x, float *y, int64_t n, unsigned long long *status,
                     void *stream);

/* Features x[i][0..5] of n Riemann problems given as float32 SoA states. */
int enzo_mlp_features(const float *rhoL, const float *uL, const float *pL, const float *rhoR,
                      const float *uR, const float *pR, double gamma, float *x, int64_t n, void *stream);

/* One training step on n samples (x[n][6], target[n], DEVICE float32): the MSE
 * loss mean((y - target)^2) goes to *loss and its gradient with respect to the
 * master parameters to grad[ENZO_MLP_PARAMS] (both overwritten; forward and
 * backward on tensor cores, BF16 operands, FP32 accumulation).  If lr > 0, an
 * Adam step (beta1 0.9, beta2 0.999, eps 1e-8, bias-corrected with the 1-based
 * step) updates master, adam_m and adam_v, and the blob is re-packed. */
int enzo_mlp_train_step(float *master, float *adam_m, float *adam_v, int32_t step, const float *x,
                        const float *target, int64_t n, float lr, float *grad, float *loss, void *blob,
                        unsigned long long *status, void *stream);

/* ---- static AMR hierarchy (Sec. 3): ghost fill from parents and siblings,
 * flux correction and projection.  A level is one enzo_patch_batch; every
 * patch also has a link giving its place in the level's global index space. */
typedef struct {
    int32_t origin[3];  /* global index (at this level) of the first active cell */
    int32_t parent;     /* index of the enclosing patch in the parent level, -1 for none */
} enzo_patch_link;

typedef struct {        /* a box of ghost cells of patch dst copied from sibling src */
    int32_t dst, src;
    int32_t lo[3], hi[3];   /* global cell box at the level, hi exclusive */
} enzo_copy_box;

typedef struct {        /* (part of) a face of a fine patch on the boundary of the refined region */
    int32_t fine;       /* fine patch index */
    int32_t dir;        /* axis of the face normal */
    int32_t side;       /* 0: low face, 1: high face */
    int32_t target;     /* coarse patch holding the coarse cells outside that part */
    int32_t lo[2], hi[2]; /* the part: coarse cells [lo, hi) along the face's two other
                             axes (a1 < a2), counted from the face's first coarse cell;
                             the whole face is [0, n_a / 2) */
} enzo_fc_face;

/* SetBoundaryValues of a refined level (Sec. 3.1): ghost cells are
 * interpolated from the parent level by SecondOrderA (Appendix A) after linear
 * interpolation in time, parent = parent_old + w (parent_new - parent_old),
 * then overwritten by copies of the siblings' active cells.  Only the ghost
 * regions listed in interp_boxes (regions no sibling covers; src unused) are
 * interpolated, since the copies replace the rest; copy_boxes list the
 * sibling copies.  parent_old and parent_new share the parent level's
 * descriptors (parent_new->patches) and differ in U.  precision ENZO_FP64: the
 * interpolation arithmetic in FP64; ENZO_FP32: in FP32 (for the FP32 path,
 * whose reconstruction reads the ghosts in FP32).  Refinement factor r = 2.
 * Gas energy (dual energy, Sec. 4.1.1): when fine->ge is non-NULL it is a sixth
 * field, interpolated and copied like the others; parent_new->ge and
 * parent_old_ge (DEVICE, the parent's ge at the start of its step) must then
 * be non-NULL too, and both NULL when fine->ge is (ENZO_ERR_ARG otherwise;
 * parent_old_ge is not read when ninterp is 0). */
int enzo_ghost_fill_level(const enzo_patch_batch *fine, const enzo_patch_link *fine_links,
                          const enzo_patch_batch *parent_new, const enzo_patch_link *parent_links,
                          double *const parent_old_U[5], const double *parent_old_ge, double w,
                          const enzo_copy_box *interp_boxes,
                          int32_t ninterp, const enzo_copy_box *copy_boxes, int32_t ncopy, int32_t precision,
                          int32_t r);

/* Flux correction (Sec. 3.4): for each listed face part of a fine patch, the
 * coarse cells just outside it get U += (dt_coarse F_coarse - mean of the fine
 * register over the r^2 fine faces) / dx_coarse on the low side (minus on the
 * high side).  F_coarse is read from the parent's all-face register, the fine
 * sums from the fine patch's boundary register.  increments != 0: the registers
 * were written by FP32-path sweeps and hold the increments the cells applied
 * (dt/dx F), and the correction is G_coarse - mean(fine sums) / r.  Parts listed
 * in one call must not share a coarse cell (the additions are unordered); a
 * caller with parts that do (concave corners of the refined region) splits
 * them over calls in the order the additions should happen.  When the batches
 * carry gas energy (coarse->ge and fine->ge both non-NULL; one alone is
 * ENZO_ERR_ARG) the registers have six components and ge is corrected with
 * the sixth, its advected flux. */
int enzo_flux_correct(const enzo_patch_batch *coarse, const enzo_patch_link *coarse_links,
                      const enzo_patch_batch *fine, const enzo_patch_link *fine_links,
                      const enzo_fc_face *faces, int32_t nface, double dt_coarse, int32_t r,
                      int32_t increments);

/* Copy between two batches of one level (a rebuild, Sec. 3.5): the cells of
 * each box (global cells at the level, hi exclusive) go from src patch
 * boxes[i].src of `src` to dst patch boxes[i].dst of `dst`, all five fields
 * (six when both batches carry gas energy; one alone is ENZO_ERR_ARG).
 * Boxes must lie in the source patch's active cells and in the destination
 * patch's stored block; boxes with the same destination must not overlap.
 * Runs on dst->stream.  ENZO_ERR_ARG on NULL arguments or nbox < 0. */
int enzo_copy_level(const enzo_patch_batch *dst, const enzo_patch_link *dst_links,
                    const enzo_patch_batch *src, const enzo_patch_link *src_links,
                    const enzo_copy_box *boxes, int32_t nbox);

/* ---- hierarchy rebuild (Sec. 3.5, 3.6) ---- */

/* Refinement criteria of Sec. 3.6, each off when its threshold is <= 0. */
typedef struct {
    double gamma;       /* ratio of specific heats (pressure of the shock criterion) */
    double slope;       /* slope: |q_{i+1} - q_{i-1}| / (2 |q_i|) > slope for q = rho or E
                           along any axis (typically 0.3) */
    double shock_dp;    /* shocks: |p_{i+1} - p_{i-1}| / min(p_{i+1}, p_{i-1}) > shock_dp
                           (0.33) with u_{i-1} - u_{i+1} > 0 along that axis ... */
    double shock_e;     /* ... and e_i / E_i > shock_e (0.1), e = E - KE */
    double mass;        /* baryon mass: rho dx^3 > mass */
    int32_t precision;  /* ENZO_FP64: every ratio formed in FP64 as written above (the
                           default of a zeroed struct); ENZO_FP32: slope and shock from
                           FP32 primitives (FP64 values rounded toward zero) compared
                           without division, |q_{i+1} - q_{i-1}| > 2 slope |q_i|,
                           |dp| > shock_dp min(p), e_i > shock_e E_i; a cell whose FP64
                           ratio lies within about 1e-6 of its threshold may then flag
                           differently.  The mass test is FP64 in both.  Other values:
                           ENZO_ERR_ARG */
} enzo_flag_params;

enum { ENZO_FLAG_SLOPE = 1, ENZO_FLAG_SHOCK = 2, ENZO_FLAG_MASS = 4 };

/* Flag the active cells of every patch of a batch (Sec. 3.6): flags[flag_off[i]
 * + (k n_y + j) n_x + i] receives the ENZO_FLAG_* bits of active cell (i, j, k)
 * of patch i (DEVICE arrays: uint8 flags, int64 flag_off[npatch]).  Neighbours
 * come from the ghost zones, which the caller fills first, or wrap for
 * ENZO_PATCH_PERIODIC patches.  Each operation is rounded once in the order
 * written (fp->precision picks FP64 or FP32), so the flags are exact functions
 * of the fields.  Uses the batch's workspace and stream.  ENZO_ERR_ARG on NULL
 * arguments or an unknown precision. */
int enzo_flag_cells(const enzo_patch_batch *b, const enzo_flag_params *fp, uint8_t *flags,
                    const int64_t *flag_off);

/* Clustering of Sec. 3.5 (Berger & Rigoutsos).  The cell-growth and
 * split rules: */
typedef struct {
    double efficiency;  /* adopt a region whose flagged fraction is >= this (0.3) ... */
    int32_t small_cells;/* ... or that holds at most this many cells (>= 1) */
    int32_t buffer;     /* flags are first grown by this many cells (Chebyshev distance,
                           inside the grid), >= 0 ... */
    int32_t margin;     /* ... and then cleared within this many cells of the grid's edge,
                           >= 0 (keeps new grids off the domain boundary or properly
                           nested in their parent) */
} enzo_cluster_params;

typedef struct {
    int32_t lo[3], hi[3];   /* half-open box of active-cell indices (x, y, z) */
} enzo_box;

/* Cover the flagged cells of one grid (HOST flags [n_z][n_y][n_x], nonzero =
 * flagged) by disjoint boxes.  The smallest box around the (grown) flags of a
 * region is adopted when efficient or small enough; otherwise it is cut in two
 * at the strongest inflection of the flag signature (a sign change of its
 * second difference, strength |change|; ties to the cut nearest the centre,
 * then the lower cut) along the longest axis, else the next longest (ties x, y,
 * z), else the longest axis is halved, and each part is processed the same
 * way, the low part first.  Host code, no GPU.  Writes at most cap boxes to the
 * HOST array boxes and the number found to *nbox; ENZO_ERR_RANGE if more than
 * cap are needed (*nbox then holds the number needed), ENZO_ERR_ARG on bad
 * arguments. */
int enzo_cluster_flags(const uint8_t *flags, const int32_t n[3], const enzo_cluster_params *cp,
                       enzo_box *boxes, int32_t cap, int32_t *nbox);

/* Projection (Sec. 3.3): every coarse cell covered by a fine patch becomes the
 * mean of its r^3 fine cells (r = 2), in every field, the gas energy too when
 * both batches carry it (one alone is ENZO_ERR_ARG). */
int enzo_project(const enzo_patch_batch *coarse, const enzo_patch_link *coarse_links,
                 const enzo_patch_batch *fine, const enzo_patch_link *fine_links, int32_t r);

/* ---- hierarchy driver (Sec. 3: EvolveLevel with subcycling; Sec. 3.5, 3.6:
 * rebuild).  The library owns a hierarchy's device state and runs its whole
 * root step: per level the ghost fill (enzo_ghost_fill_level from the parent,
 * interpolated in time, then the sibling copies; enzo_ghost_fill_boundary on a
 * root with external boundaries), the level's CFL timestep (capped at its
 * parent's time), a copy of the state at the start of the step for a level
 * with children, the three sweeps in alternating order recording flux
 * registers, then, for a level with children, the ghost fill at the new time,
 * the finer level advanced to this level's time by the same rules, flux
 * correction in the order of its face parts, projection, and optionally a
 * rebuild.  The plans (sibling copy boxes, interpolated ghost regions,
 * correction face parts in waves) are built on the host at creation and again
 * for every rebuilt level.  All calls are host-synchronous where a host value
 * is needed (every level CFL, a rebuild's flags) and otherwise queue work on
 * the hierarchy's stream. */
typedef struct enzo_hierarchy enzo_hierarchy;   /* opaque */

typedef struct {
    int32_t npatch;         /* patches of the level (>= 0; exactly 1 on the root level) */
    const int32_t *n;       /* HOST [npatch][3] active cells per axis (>= 1; even below the root) */
    const int32_t *origin;  /* HOST [npatch][3] global index at this level of the first active
                               cell (even below the root: patches cover whole parent cells) */
    const int32_t *parent;  /* HOST [npatch] index of the enclosing patch in level l-1, -1 on
                               level 0 */
} enzo_level_layout;

/* Device memory for a hierarchy: alloc returns a DEVICE block of at least
 * `bytes` (256-byte aligned) or NULL; release frees it.  ctx is passed
 * through.  A NULL allocator (or NULL members) selects cudaMalloc / cudaFree. */
typedef void *(*enzo_alloc_fn)(size_t bytes, void *ctx);
typedef void (*enzo_free_fn)(void *ptr, void *ctx);
typedef struct {
    enzo_alloc_fn alloc;
    enzo_free_fn release;
    void *ctx;
} enzo_allocator;

/* Rebuild rules (Sec. 3.5, 3.6): cells flagged by `flag` (enzo_flag_cells) are
 * clustered per patch by `cluster` (enzo_cluster_flags; its margin member is
 * replaced by root_margin on level 0 and by nest below, which keeps new grids
 * off the domain boundary or properly nested). */
typedef struct {
    enzo_flag_params flag;
    enzo_cluster_params cluster;
    int32_t root_margin;    /* typically 3 */
    int32_t nest;           /* typically 1 */
} enzo_rebuild_params;

/* Build a hierarchy of nlevel levels (refinement factor 2 between levels).
 * Level l has cell width root_dx / 2^l.  nfields: 5, or 6 with the gas energy
 * of the dual-energy option (then carried by every operation; sweeps need
 * ENZO_OPT_DUAL).  root_bc: HOST bc[3] (ENZO_BC_*) of a root whose ghosts are
 * filled before each step, or NULL for a periodic root that wraps inside its
 * sweeps (then level 1 must stay 3 root cells from the domain boundary:
 * ENZO_ERR_RANGE otherwise).  stream: cudaStream_t of every operation.
 * Fields start at zero: fill them through enzo_hierarchy_level's batch (e.g.
 * enzo_unpack_active or copies into U).  *out receives the hierarchy.
 * ENZO_ERR_ARG on inconsistent layouts (parent out of range, odd sizes or
 * origins below the root), ENZO_ERR_CUDA when memory runs out. */
int enzo_hierarchy_create(const enzo_level_layout *levels, int32_t nlevel, double root_dx, int32_t nfields,
                          const int32_t *root_bc, void *stream, const enzo_allocator *allocator,
                          enzo_hierarchy **out);

/* Free a hierarchy's device memory (after synchronising its stream). */
int enzo_hierarchy_destroy(enzo_hierarchy *h);

/* Number of levels. */
int enzo_hierarchy_nlevel(const enzo_hierarchy *h);

/* One level's state, owned by the hierarchy: valid until that level is
 * rebuilt (generation then changes) or the hierarchy is destroyed. */
typedef struct {
    enzo_patch_batch batch;         /* its fields, descriptors, workspace, status, registers
                                       (stream: the hierarchy's) */
    const enzo_patch_link *links;   /* DEVICE [npatch] */
    const enzo_patch *table;        /* HOST [npatch] copy of the descriptors */
    const int32_t *n, *origin, *parent;   /* HOST layout, as in enzo_level_layout */
    double dx;                      /* cell width */
    double t;                       /* the level's time */
    int64_t cells;                  /* active cells */
    int64_t freg_len;               /* doubles in batch.freg */
    uint64_t generation;            /* the hierarchy's rebuild counter */
} enzo_level_info;
int enzo_hierarchy_level(const enzo_hierarchy *h, int32_t level, enzo_level_info *info);

/* One root step: dt_0 = the root's CFL timestep (rule of `cfl`, NULL: p), then
 * EvolveLevel from level 0 to t + dt_0 with the sweep parameters p.  rb: NULL
 * (static hierarchy) or the rules of a rebuild after every step of a level with
 * children (after flux correction and projection), which replaces every finer
 * level.  *dt0_out (may be NULL) receives dt_0.  The (level, dt) of every level
 * step is appended to the hierarchy's log (enzo_hierarchy_take_log).  Any
 * ENZO_ERR_* of a library call it makes is returned (the state is then
 * undefined). */
int enzo_hierarchy_root_step(enzo_hierarchy *h, const enzo_params *p, const enzo_params *cfl,
                             const enzo_rebuild_params *rb, double *dt0_out);

/* As enzo_hierarchy_root_step with the root's step ending at t_end (> the
 * root's time) instead of its CFL timestep, e.g. to land on an output time; the
 * caller keeps t_end - t within the root's CFL limit. */
int enzo_hierarchy_step_to(enzo_hierarchy *h, double t_end, const enzo_params *p, const enzo_params *cfl,
                           const enzo_rebuild_params *rb);

/* Rebuild levels level+1, level+2, ... now (Sec. 3.5, 3.6): level `level`'s
 * ghosts are filled, its cells flagged and clustered, and each new patch is
 * interpolated from its parent (FP64, SecondOrderA) and overwritten by the old
 * patches of its level where they overlap; a level whose grids come out
 * unchanged is kept.  HOST boxes[nbox][7] receives the new grids of level+1 as
 * (parent, lo[3], hi[3]) in level-`level` cells, *nbox their number
 * (ENZO_ERR_RANGE, after the rebuild, when more than cap). */
int enzo_hierarchy_rebuild(enzo_hierarchy *h, int32_t level, const enzo_rebuild_params *rb, int32_t *boxes,
                           int32_t cap, int32_t *nbox);

/* Move the step log into HOST levels[] / dts[] (cap entries) and clear it;
 * *n receives the number of entries (ENZO_ERR_RANGE, log kept, when > cap). */
int enzo_hierarchy_take_log(enzo_hierarchy *h, int32_t *levels, double *dts, int32_t cap, int32_t *n);

/* Device time per operation kind, from CUDA events around each operation on
 * the hierarchy's stream while timing is on: ms[ENZO_HOP_*] (HOST, may be
 * NULL; synchronises the stream).  *cell_updates (may be NULL): active cells
 * swept (one per cell per level step) since creation.  enable: 1 clears the
 * times and turns timing on, 0 clears and turns it off, -1 leaves it as it is. */
enum {
    ENZO_HOP_GHOST_FILL = 0, ENZO_HOP_CFL = 1, ENZO_HOP_SAVE_OLD = 2, ENZO_HOP_SWEEPS = 3,
    ENZO_HOP_CORRECT_PROJECT = 4, ENZO_HOP_REBUILD = 5, ENZO_HOP_COUNT = 6
};
int enzo_hierarchy_timing(enzo_hierarchy *h, int32_t enable, double ms[ENZO_HOP_COUNT], int64_t *cell_updates);

/* The driver's plans on their own (host code, no GPU).  enzo_plan_level: for a
 * level's layout (HOST n[npatch][3], origin[npatch][3]), the sibling copy boxes
 * (every intersection of a patch's ghost-extended box with another patch's
 * active box, by destination then source) and the ghost regions to interpolate
 * (of the 26 around each patch, z slowest, then y, x, each -1, 0, 1: those not
 * lying wholly in one sibling's active box; dst = src = the patch).
 * enzo_plan_correction: the flux-correction face parts of a coarse level
 * against its fine level (Sec. 3.4) in the order (fine patch, axis, side,
 * coarse patch), and for each a wave: parts in one wave share no coarse cell,
 * and a part that shares cells with earlier ones comes in a later wave.
 * Outputs go to HOST arrays of cap entries; the counts are written first
 * (ENZO_ERR_RANGE when they exceed the capacity). */
int enzo_plan_level(const int32_t *n, const int32_t *origin, int32_t npatch, enzo_copy_box *sib, int32_t sib_cap,
                    int32_t *nsib, enzo_copy_box *itp, int32_t itp_cap, int32_t *nitp);
int enzo_plan_correction(const int32_t *fine_n, const int32_t *fine_origin, int32_t nfine, const int32_t *coarse_n,
                         const int32_t *coarse_origin, int32_t ncoarse, enzo_fc_face *parts, int32_t *wave,
                         int32_t cap, int32_t *nparts);

/* ---- measurement helper (not part of the method) ---- */

/* Throughput probe of the FP64 pipe, the denominator of the FP64 sweep's ALU
 * roofline.  Launches ENZO_PROBE_BLOCKS_PER_SM x (SM count) blocks of 256
 * threads on `stream` (a cudaStream_t); each thread runs 8 independent chains
 * of n steps of one operation: ENZO_PROBE_DFMA x = fma(x, a, b), _DADD x + b,
 * _DMUL x * a, _DSQRT sqrt(x + b), _DDIV a / (x + b) (IEEE division and square
 * root, as the FP64 path executes them).  *ops (HOST) receives the number of
 * operations launched; the caller times the launch (CUDA events) and divides.
 * sink: a DEVICE array of at least (blocks + 1) doubles the kernel may write.
 * ENZO_ERR_ARG on a bad op, n < 1 or n > 2^30, or NULL pointers. */
enum { ENZO_PROBE_DFMA = 0, ENZO_PROBE_DADD = 1, ENZO_PROBE_DMUL = 2, ENZO_PROBE_DSQRT = 3, ENZO_PROBE_DDIV = 4 };
#define ENZO_PROBE_BLOCKS_PER_SM 4
int enzo_probe_fp64(int32_t op, int64_t n, double *sink, int64_t *ops, void *stream);

/* Text for an ENZO_ERR_* code (static storage). */
const char *enzo_strerror(int code);

/* Number of kernels the library launched in this process since load. */
unsigned long long enzo_launch_count(void);

#ifdef __cplusplus
}
#endif
#endif /* ENZO_PPM_H */
