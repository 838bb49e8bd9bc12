/*
 * lbm.h - C ABI of the GB300 (sm_103a) anisotropic-equilibrium BGK lattice Boltzmann library.
 *
 * Method: Kruger, Weinmiller, Latz, Danner, "Lattice Boltzmann Methods with Anisotropic
 * Equilibrium Distributions". One time step is the fully discrete BGK LBE of Eq. (LBE_BGK),
 *     f_i(x + c_i, t + 1) = f_i(x, t) + (feq_i(x, t) - f_i(x, t)) / tau,
 * with the third-order discrete anisotropic equilibrium of Eq. (3rd_order_equilibrium)/(feq_i):
 *     feq_i = w_i rho [1 + u.c_i/cs2 + ((u.c_i)^2 - cs2 |u|^2 + h_i)/(2 cs2^2)
 *                      + ((u.c_i)^3 - 3 cs2 |u|^2 u.c_i + 3 h_i u.c_i - 6 cs2 c_i.K~.u)/(6 cs2^3)],
 *     K~ = Theta - cs2 I (Eq. K-term with Theta = cs2 A^{-1}), h_i = c_i.K~.c_i - cs2 tr K~,
 * on the D2Q9, D3Q19 and D3Q27 velocity sets (Appendix C; cs2 = 1/3). The second moment of the
 * equilibrium is rho (Theta + u u) (Appendix E), so Theta is the anisotropy tensor in lattice
 * units; Theta = cs2 I is standard BGK. Walls are half-way bounce-back on a solid mask (the paper
 * names bounce-back only as future work, Sec. 5; the textbook rule is used).
 *
 * Conventions for every call:
 *   - Cells are indexed n = x + nx*(y + ny*z); D2Q9 requires nz == 1.
 *   - Field buffers are DEVICE pointers owned by the caller, element type double when the
 *     context stores FP64 and float otherwise. Layouts: rho [N]; u [d][N]; Pi [d(d+1)/2][N]
 *     ordered xx, yy, (zz), xy, (xz, yz). The velocity u is the paper's lattice velocity s.
 *   - Theta is a HOST array of d*d doubles, row-major, symmetric positive definite.
 *   - Every call is issued on the context's stream and returns without synchronising unless it
 *     says so; an asynchronous CUDA error surfaces at the next synchronising call.
 *   - Return value: LBM_OK (0) or a negative lbm_status. Nothing throws across this boundary.
 *     lbm_last_error() gives a one-line description of the last failure of a context.
 *   - The state visible to the user after lbm_init followed by lbm_step(n) is the pre-collision
 *     population set f(n); lbm_moments and lbm_populations report it.
 */
#ifndef LBM_H
#define LBM_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct lbm_ctx lbm_ctx;

/* Velocity sets (Appendix C). */
enum lbm_lattice { LBM_D2Q9 = 9, LBM_D3Q19 = 19, LBM_D3Q27 = 27 };

/* Population storage. Arithmetic is FP32 except in LBM_FP64. Shifted forms store
 * f_i - r_i with r_i = feq_i(rho0, u = 0; Theta) = w_i rho0 (1 + h_i/(2 cs2^2)), the rest
 * equilibrium (equals w_i rho0 when Theta = cs2 I). LBM_FP16_WSHIFTED stores f_i - w_i rho0 in
 * FP16, the shift by the lattice weights alone: when Theta != cs2 I its stored values carry the
 * offset r_i - w_i rho0 as well, which costs FP16 precision; it is kept as the comparison
 * (ablation) for LBM_FP16_SHIFTED, runs one cell per thread, and is not meant for production. */
enum lbm_storage { LBM_FP32 = 0, LBM_FP64 = 1, LBM_FP32_SHIFTED = 2, LBM_FP16_SHIFTED = 3, LBM_FP16_WSHIFTED = 4 };

/* Streaming schemes: two arrays in pull form, or one array in the AA pattern (in place). */
enum lbm_scheme { LBM_PULL2 = 0, LBM_AA = 1 };

enum lbm_status {
    LBM_OK = 0,
    LBM_ERR_INVALID_ARG = -1, /* bad pointer, size, enum or option */
    LBM_ERR_NOT_SPD = -2,     /* Theta not symmetric positive definite */
    LBM_ERR_BAD_TAU = -3,     /* tau <= 1/2 (non-positive viscosity, Sec. 3) */
    LBM_ERR_OOM = -4,         /* device or host allocation failed */
    LBM_ERR_CUDA = -5,        /* a CUDA runtime call or kernel launch failed */
    LBM_ERR_UNSTABLE = -6,    /* a cell reached rho <= 0 or a non-finite value */
    LBM_ERR_NO_FORWARD = -7,  /* adjoint asked for n steps but n steps were not run since init */
    LBM_ERR_TIMEOUT = -8,     /* reserved for bounded device waits (none are used) */
    LBM_ERR_STATE = -9,       /* call out of order (e.g. step before init) */
    LBM_ERR_HALO = -10        /* the halo-exchange callback of a z-slab context failed */
};

/* Allocator hooks for library-owned device memory (populations, adjoint buffers, checkpoints).
 * alloc returns a device pointer of at least `bytes` bytes, 256-byte aligned, or NULL. */
typedef void* (*lbm_alloc_fn)(size_t bytes, void* user);
typedef void (*lbm_free_fn)(void* ptr, void* user);

/* Halo exchange of a z-slab context (see "Z-slab decomposition" below). The library calls it
 * after every kernel that writes a [q][N] array whose ghost planes a later kernel reads, with
 * `array` that array (library-owned device memory) and `kind` LBM_HALO_POPULATIONS or
 * LBM_HALO_ADJOINT. On return the two ghost planes of `array` must hold the neighbouring slabs'
 * boundary planes (lbm_halo_pack / lbm_halo_unpack), ordered before the next kernel on the
 * context's stream. Return 0 on success; anything else stops the call with LBM_ERR_HALO. */
typedef int (*lbm_halo_fn)(struct lbm_ctx* ctx, int kind, void* array, void* user);
enum lbm_halo_kind { LBM_HALO_POPULATIONS = 0, LBM_HALO_ADJOINT = 1 };

typedef struct {
    int storage;              /* enum lbm_storage; lbm_options_default (and a NULL opt) select
                                 LBM_FP32_SHIFTED; a zeroed struct selects plain LBM_FP32, which
                                 rounds f ~ w_i instead of f - r_i ~ O(u) and loses about an
                                 order of magnitude of velocity accuracy at the same speed */
    int scheme;               /* enum lbm_scheme; default LBM_PULL2 */
    int order;                /* 3 (default, also when 0) or 2: equilibrium truncation order */
    double rho0;              /* reference density of the shifted forms; 0 -> 1.0 */
    int check_every;          /* > 0: lbm_step synchronises and checks stability every k steps */
    int use_graphs;           /* 0: CUDA graphs for small grids, 1: always, -1: never */
    lbm_alloc_fn alloc;       /* NULL: cudaMalloc */
    lbm_free_fn free;         /* must be set together with alloc */
    void* alloc_user;         /* passed to alloc/free */
    void* stream;             /* cudaStream_t for every launch; NULL: the legacy default stream */
    size_t adjoint_mem_limit; /* bytes of device memory for saved states (checkpoints and the
                                 states of one segment); checkpoints beyond it go to pinned host
                                 memory, segments beyond it are recomputed in two levels;
                                 0: free device memory minus a margin */
    int z_halo;               /* 1: the context is one z-slab of a larger periodic box (below);
                                 0: a whole periodic box (default) */
    lbm_halo_fn halo;         /* z-slab exchange callback; NULL: the slab is the whole box in z
                                 and its ghost planes are filled from its own boundary planes */
    void* halo_user;          /* passed to halo */
} lbm_options;

/* Fill *opt with the defaults (all zero except as documented above). */
int lbm_options_default(lbm_options* opt);

/* Create a context for an nx*ny*nz lattice with relaxation time tau (Eq. LBE_BGK; kinematic
 * viscosity (tau - 1/2) Theta, Eq. NSprefinal2) and anisotropy Theta (host, d*d).
 * solid_mask: N bytes, nonzero = solid cell, host or device memory (detected), or NULL for an
 * all-fluid periodic box. Boundaries are periodic on every axis; walls come only from the mask.
 * Synchronises. On success *out owns the context; release it with lbm_destroy. */
int lbm_create(lbm_ctx** out, int lattice, int nx, int ny, int nz, double tau, const double* Theta,
               const uint8_t* solid_mask);
int lbm_create_ex(lbm_ctx** out, int lattice, int nx, int ny, int nz, double tau, const double* Theta,
                  const uint8_t* solid_mask, const lbm_options* opt);
void lbm_destroy(lbm_ctx* ctx);

/* Change tau or Theta of an existing context (same validation as lbm_create). The current
 * populations are discarded: call lbm_init before the next lbm_step (LBM_ERR_STATE otherwise). */
int lbm_set_params(lbm_ctx* ctx, double tau, const double* Theta);

/* f(0) = feq(rho, u) at every fluid cell (Sec. 4 initialises from the macroscopic fields).
 * rho: device [N] or NULL (uniform rho0); u: device [d][N] or NULL (at rest). Values at solid
 * cells are ignored. Resets the step counter; the fields are kept for lbm_adjoint. */
int lbm_init(lbm_ctx* ctx, const void* rho, const void* u);

/* Advance n >= 0 time steps of Eq. LBE_BGK: one fused stream + collide kernel per step. */
int lbm_step(lbm_ctx* ctx, int n);

/* Macroscopic fields of f(t): rho = sum f_i, u = sum f_i c_i / rho (Eqs. a0discrete_f,
 * a1discrete_f), Pi_ab = sum f_i c_ia c_ib. Any pointer may be NULL. Solid cells get 0. */
int lbm_moments(lbm_ctx* ctx, void* rho, void* u, void* Pi);

/* Pre-collision populations f_i(x, t) into device [q][N], in the library's direction order
 * (lbm_lattice_info). Solid cells get 0. */
int lbm_populations(lbm_ctx* ctx, void* f);

/* FP64 totals over fluid cells: mass = sum rho, momentum[a] = sum rho u_a (host outputs; either
 * may be NULL). Deterministic order. Synchronises. Returns LBM_ERR_UNSTABLE if any fluid cell
 * has rho <= 0 or a non-finite moment. */
int lbm_totals(lbm_ctx* ctx, double* mass, double* momentum);

/* Keep the stored state at every multiple of checkpoint_every steps of the current trajectory
 * (from lbm_init on; 0 stops recording), in device memory while adjoint_mem_limit allows and in
 * pinned host memory beyond. A following lbm_adjoint with the same checkpoint_every then
 * recomputes only inside segments instead of re-running the whole forward pass. Call it before
 * lbm_init or right after it (step 0). */
int lbm_record_checkpoints(lbm_ctx* ctx, int checkpoint_every);

/* Discrete adjoint of f(0) = feq(rho0, u0) -> f(n) -> u(n) for a loss L(u(n)) with
 * loss_grad = dL/du(n) (device [d][N], field type). Requires exactly n steps since the last
 * lbm_init (else LBM_ERR_NO_FORWARD). Works backward in segments of checkpoint_every steps
 * (0: the recorded interval, else about sqrt(n)): each segment is recomputed from its checkpoint
 * (recorded by lbm_record_checkpoints, or taken here by a forward pass from the initial fields)
 * and then swept by one adjoint kernel per step; when the segment's states do not all fit on
 * the device it is recomputed in sub-segments (the first pass keeps their starts and the last
 * one's states, the others are recomputed again in their turn). Host-memory checkpoints are
 * copied back on a second stream one segment ahead of use when one more state fits on the
 * device. Leaves f(n) in place. Results are read with lbm_gradients. The working set (two lambda
 * arrays, the segment states) is allocated by the first call and kept for later calls (an
 * optimisation loop pays for it once) until lbm_adjoint_release or lbm_destroy. Synchronises. */
int lbm_adjoint(lbm_ctx* ctx, const void* loss_grad, int n, int checkpoint_every);

/* Plan of the last lbm_adjoint: sub_segment = the longest sub-segment of a full segment when
 * segments are recomputed in sub-segments (the states of fewer than checkpoint_every steps fit),
 * else checkpoint_every (flat recompute); prefetched = host checkpoints copied back ahead of use.
 * Either pointer may be NULL. No counterpart in the paper (memory plan of the checkpointed
 * adjoint). */
int lbm_adjoint_info(const lbm_ctx* ctx, int* sub_segment, int* prefetched);

/* The recompute plan lbm_adjoint follows for one segment of `len` steps when `working` state
 * buffers are free besides the segment start: *count sub-segment starts s_0 = 0 < ... < s_m < len
 * are written to starts[0 .. *count - 1] (capacity entries available; *count = 1, starts = {0}, when
 * the segment is recomputed flat, i.e. len - 1 <= working). The first recompute pass keeps the
 * states s_1 .. s_(m-1) and every state of the last sub-segment [s_m, len); each earlier
 * sub-segment, at most len - s_m + 1 steps, is recomputed from its start into the last one's
 * buffers when its turn comes; the plan costs 2 len - 2 - working recompute steps (flat: len - 1).
 * Host computation only, no context or device. Returns LBM_ERR_OOM when no such plan fits in
 * `working` buffers, LBM_ERR_INVALID_ARG for len < 1, working < 0, a null pointer or too small a
 * capacity. No counterpart in the paper (memory plan of the checkpointed adjoint). */
int lbm_adjoint_plan(int len, int working, int* starts, int capacity, int* count);

/* Free the adjoint's large working set (the lambda arrays and the segment states) that
 * lbm_adjoint keeps between calls; du0 and the gradients of the last call stay readable.
 * Synchronises. No counterpart in the paper (memory management of the checkpointed adjoint). */
int lbm_adjoint_release(lbm_ctx* ctx);

/* Gradients of the last lbm_adjoint: dTheta (host, 3 values in 2D: xx, yy, xy; 6 in 3D:
 * xx, yy, zz, xy, xz, yz; an off-diagonal entry is dL/dTheta_ab + dL/dTheta_ba), dtau (host),
 * du0 (device [d][N], field type). Any pointer may be NULL. Synchronises. */
int lbm_gradients(lbm_ctx* ctx, double* dTheta, double* dtau, void* du0);

/* Raw state for save/resume: a header plus the stored populations. dst/src may be host or
 * device memory. lbm_state_bytes gives the size. Restoring into a context created with the same
 * lattice, size, storage and scheme reproduces the run bit for bit. */
int lbm_state_bytes(const lbm_ctx* ctx, size_t* bytes);
int lbm_get_state(lbm_ctx* ctx, void* dst, size_t bytes);
int lbm_set_state(lbm_ctx* ctx, const void* src, size_t bytes);

/* Steps taken since the last lbm_init (or restored with the state). */
int lbm_steps_done(const lbm_ctx* ctx, long long* steps);

/* Wait for the context's stream; reports asynchronous CUDA errors. */
int lbm_sync(lbm_ctx* ctx);

/* The library's velocity set: c [q][3] (ints) and w [q] (host). Returns q, or a negative
 * status for an unknown lattice. Directions come in opposite pairs: 0 is rest, 2k+1 and 2k+2
 * are opposite. */
int lbm_lattice_info(int lattice, int* c, double* w);

/* Bytes of library-owned device memory held by the context. */
int lbm_device_bytes(const lbm_ctx* ctx, size_t* bytes);

/* Kernel launches issued by this context since creation (all kinds). */
int lbm_launch_count(const lbm_ctx* ctx, long long* launches);

/* ---------------------------------------------------------------------------------------------
 * Anisotropic advection-diffusion of a scalar phi (Sec. 1 and Sec. 5 name the transfer of the
 * anisotropic equilibrium to advection-diffusion; the paper gives no equations for it).
 * Populations g_i with phi = sum g_i relax by BGK (Eq. LBE_BGK) towards the equilibrium of
 * Eq. (3rd_order_equilibrium) with rho -> phi and u the PRESCRIBED advecting velocity, so
 * sum geq = phi, sum geq c = phi u, sum geq c c = phi (Theta + u u). Only phi is conserved; the
 * Chapman-Enskog limit (Sec. 3 with rho -> phi) is d_t phi + div(phi u) = div(D grad phi) with
 * the anisotropic diffusion tensor D = (tau - 1/2) Theta (exact for a uniform u: the covariance
 * of a concentration blob grows by 2 D per step). Walls (half-way bounce-back on the mask) are
 * zero-flux boundaries.
 *
 * A scalar context is an lbm_ctx made by lbm_ade_create; these calls apply to it unchanged:
 *   lbm_init(ctx, phi, NULL)  g(0) = geq(phi, u) with the current advecting velocity; phi device
 *                             [N] or NULL (uniform rho0); u must be NULL (LBM_ERR_INVALID_ARG)
 *   lbm_step, lbm_populations, lbm_state_bytes / lbm_get_state / lbm_set_state (a state keeps
 *   its kind and restores only into a context of the same kind), lbm_steps_done, lbm_sync,
 *   lbm_set_params, lbm_device_bytes, lbm_launch_count, lbm_destroy;
 *   lbm_moments(ctx, phi, j_over_phi, Pi)  rho slot = phi; u slot = sum g c / phi (the scalar's
 *                             total flux over phi); Pi = sum g c c;
 *   lbm_totals(ctx, &total, flux)  total = sum phi, flux = sum g c over fluid cells; fails with
 *                             LBM_ERR_UNSTABLE only for non-finite values (phi <= 0 is allowed).
 * lbm_adjoint, lbm_record_checkpoints and lbm_gradients return LBM_ERR_INVALID_ARG on it.
 * opt->rho0 is the reference phi0 of the shifted storage forms (choose it near the typical phi
 * for FP16 storage); check_every flags non-finite phi only.
 * ------------------------------------------------------------------------------------------- */

/* Same arguments, validation and ownership as lbm_create_ex. The advecting velocity starts at 0
 * (pure anisotropic diffusion). */
int lbm_ade_create(lbm_ctx** out, int lattice, int nx, int ny, int nz, double tau, const double* Theta,
                   const uint8_t* solid_mask, const lbm_options* opt);

/* Set the advecting velocity: u = a [d][N] field (device or host, field type; copied on the
 * context's stream, values at solid cells ignored), or u_const = d host doubles (a uniform
 * velocity), or both NULL (u = 0, no velocity reads in the step kernel). Both non-NULL, a
 * non-finite constant or a flow context give LBM_ERR_INVALID_ARG. Takes effect from the next
 * lbm_step or lbm_init; the populations are kept, so the velocity may change between steps. */
int lbm_ade_set_velocity(lbm_ctx* ctx, const void* u, const double* u_const);

/* The context-owned advecting-velocity field (device [d][N], field type) for in-place updates,
 * e.g. lbm_moments(flow_ctx, NULL, *u, NULL) of a flow context with the same field type couples
 * the scalar to a flow without a copy. Allocates the field on first use (holding the current
 * velocity, zeros if it was 0) and makes the step read it. The pointer stays valid until
 * lbm_destroy; writes on other streams must be ordered before the next lbm_step. */
int lbm_ade_velocity(lbm_ctx* ctx, void** u);

/* ---------------------------------------------------------------------------------------------
 * Z-slab decomposition. Streaming (Eq. LBE_BGK) moves each population one lattice link per step,
 * so a box split into slabs along z needs, per step, only the populations with c_z = +-1 of the
 * two planes next to each cut (5 directions per plane for D3Q19, 9 for D3Q27); the reverse
 * streaming of the adjoint needs the same planes of lambda with the opposite c_z. A context
 * created with opt->z_halo = 1 holds one slab: `nz` interior planes plus one ghost plane below
 * (stored plane 0) and one above (stored plane nz + 1), i.e. N = nx*ny*(nz + 2) stored cells.
 * Every field buffer of such a context (rho, u, Pi, populations, loss_grad, du0, the advecting
 * velocity) and the solid mask span all N stored cells; kernels read and write the interior
 * planes only (ghost entries of outputs are left unchanged, of inputs ignored), and the mask's
 * ghost planes give the solidity of the neighbouring slabs' boundary planes. Totals and
 * gradients cover the slab's interior; a sharded run sums them over the slabs (FP64).
 * Restrictions: D3Q19 or D3Q27, the two-array pull scheme, flow contexts (LBM_ERR_INVALID_ARG
 * otherwise); CUDA graphs are not used. All slabs of one box must run the same sequence of
 * calls (same n, checkpoint_every and adjoint plan: give them the same adjoint_mem_limit), so
 * that their halo callbacks pair up.
 * ------------------------------------------------------------------------------------------- */

/* Bytes of one packed halo plane of `kind` (directions x nx*ny elements; populations in the
 * storage type, lambda in the field type). LBM_ERR_INVALID_ARG for a context that is not a slab. */
int lbm_halo_bytes(const lbm_ctx* ctx, int kind, size_t* bytes);

/* Pack the boundary plane that the neighbour on `side` needs (side 0: the lowest interior plane,
 * sent to the slab below; side 1: the highest, sent to the slab above) from `array` (the device
 * [q][N] array given to the callback) into the device buffer `buf` of lbm_halo_bytes bytes:
 * populations with c_z = -1 (side 0) / +1 (side 1), lambda with c_z = +1 (side 0) / -1 (side 1),
 * in increasing direction order, each an nx*ny plane. Asynchronous on the context's stream. */
int lbm_halo_pack(lbm_ctx* ctx, int kind, int side, const void* array, void* buf);

/* Unpack a neighbour's packed plane into the ghost plane on `side` of `array` (side 0: the ghost
 * plane below, filled from the lower slab's side-1 pack; side 1: the ghost plane above, from the
 * upper slab's side-0 pack). Asynchronous on the context's stream. */
int lbm_halo_unpack(lbm_ctx* ctx, int kind, int side, void* array, const void* buf);

/* FP64 totals of a caller-owned population array with no device allocation: for callers that
 * cannot call cudaMalloc, cudaFree or any allocating routine where they need the totals (code
 * under an external memory manager that owns every device byte, code that must not synchronise
 * the device through an allocation, plug-ins that only receive pointers to existing buffers).
 * The paper has no counterpart; it is the block-partial reduction of lbm_totals.
 *   f       device [q][N] populations f_i(x) in the library's direction order, float or (fp64 != 0)
 *           double, e.g. the output of lbm_populations (zeros at solid cells add nothing)
 *   totals  device double[4]: sum f, sum f c_x, sum f c_y, sum f c_z (0 in 2D)
 *   stream  cudaStream_t (NULL: legacy default stream); the call is asynchronous on it.
 * The partial sums live in one fixed __device__ array of 1216 records x 4 doubles (38,912 bytes)
 * that every GPU loading the library holds until the process exits; every call writes each
 * record it reads, so nothing needs clearing between calls, and all calls share the array:
 * calls that overlap on the GPU (other streams, other host threads) race on it. The first call
 * on a device looks up the array's device address (cudaGetSymbolAddress) and caches it for the
 * life of the process; make that first call outside any stream capture, and do not call this
 * entry point again after a cudaDeviceReset of that device (the cached address would be stale).
 * Any N up to 2^31 - 1 cells fits; larger sizes,
 * an unknown lattice, nz != 1 for D2Q9 or null pointers return LBM_ERR_INVALID_ARG. */
int lbm_totals_noalloc(int lattice, int nx, int ny, int nz, int fp64, const void* f, double* totals, void* stream);

const char* lbm_status_string(int status);
const char* lbm_last_error(const lbm_ctx* ctx);

#ifdef __cplusplus
}
#endif
#endif /* LBM_H */
