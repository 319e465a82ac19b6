/*
 * lbm.h -- C ABI of the GB300 MRT lattice Boltzmann library (liblbm.so).
 *
 * The library runs the fused multiple-relaxation-time (MRT) lattice Boltzmann time step of the
 * He-Luo D3Q19 model (and its D2Q9 and D3Q15 counterparts) on one NVIDIA GPU, forming the strain-rate
 * tensor S at every node by either of the two routes compared by Zhang, Huang, Wang and Shi,
 * "The computation of strain rate tensor in multiple-relaxation-time lattice Boltzmann model"
 * (arXiv:1704.07559):
 *   LBM_YU    Yu's formula, eq. (LuoS): S from six non-equilibrium moments;
 *   LBM_CHAI  Chai's formula, eq. (ChaiS): S from the q non-equilibrium distributions,
 *             -sum_i c_i c_i (T^-1 L T f_neq)_i / (2 rho0 cs^2).
 * On D2Q9 and D3Q15, LBM_YU selects the Yu-type formula that the procedure of Sec. 5.4 derives
 * from Chai's formula for that lattice's moment basis.
 * S feeds a strain-rate-dependent relaxation time (Smagorinsky eddy viscosity or a power-law
 * fluid) inside the same step.
 *
 * Conventions shared by every call
 *  - Lattice units: delta_x = delta_t = 1, cs^2 = 1/3, nu = (tau - 1/2)/3.
 *  - Populations are the delta-rho form of Sec. 2, eq. (edf): sum_i f_i = delta rho.  They live
 *    in two caller-owned device buffers ("A" and "B"), each holding q population arrays of
 *    `stride` elements (lbm_layout), element (i, node) at i*stride + node, node =
 *    (z*ny + y)*nx + x.  The element type is the storage precision: double (LBM_FP64), float
 *    (LBM_FP32), IEEE half (LBM_FP16S) or bfloat16 (LBM_BF16S).  The arithmetic is double for
 *    LBM_FP64 and float for the other three ("compute type" below).
 *  - The buffer most recently written holds the post-collision populations f* of the last step.
 *    Read-outs (lbm_strain_rate, lbm_macroscopic, lbm_sums) report the pre-collision state that
 *    the next step sees, obtained by pulling f_i(x) = f*_i(x - c_i) with the boundary rules.
 *  - Fields passed in or out are dense component-major arrays: component c of node n at c*N + n,
 *    N = nx*ny*nz.  Strain components are xx, yy, zz, xy, yz, xz in 3D and xx, yy, xy in 2D.
 *  - Faces are numbered -x, +x, -y, +y, -z, +z.  Opposite faces must both be periodic or both
 *    not (and both LBM_HALO, only on z).  A wall is halfway bounce-back; a moving wall ("lid") adds 2 w_i rho0 (c_i . u_w)/cs^2
 *    to the population it reflects; a population that leaves through an edge or corner where
 *    two non-periodic faces meet is reflected without the moving-wall term.
 *  - All calls are asynchronous on the bound stream unless stated otherwise, return LBM_OK or a
 *    negative status, never abort, and leave a message for lbm_last_error.
 *  - A context is not thread-safe: calls on one context must not run concurrently.
 */
#ifndef LBM_H
#define LBM_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* status codes */
#define LBM_OK 0
#define LBM_ERR_ARG -1       /* invalid argument: nothing was done */
#define LBM_ERR_CUDA -2      /* a CUDA runtime call or kernel launch failed */
#define LBM_ERR_NOMEM -3     /* the library's own small allocation failed */
#define LBM_ERR_NONFINITE -4 /* a global sum came back NaN or infinite */
#define LBM_ERR_STATE -5     /* call out of order (e.g. lbm_step before lbm_bind) */
#define LBM_ERR_DRIFT -6     /* the watchdog found the conserved totals off their balance */

/* lattices (the value is q) */
#define LBM_D2Q9 9
#define LBM_D3Q15 15 /* d'Humieres 15-moment basis (the paper names the lattice, prints no table) */
#define LBM_D3Q19 19

/* population storage precision */
#define LBM_FP64 0
#define LBM_FP32 1
#define LBM_FP16S 2 /* IEEE binary16 storage of the delta-rho form, float arithmetic */
#define LBM_BF16S 3 /* bfloat16 storage of the delta-rho form, float arithmetic */

/* closures for the viscous relaxation rate s_nu = 1/tau */
#define LBM_NEWTON 0   /* tau fixed by the rates given to lbm_create */
#define LBM_SMAG 1     /* tau = tau0 + 3 Cs^2 |S| (filter width 1) */
#define LBM_POWERLAW 2 /* tau = 1/2 + 3 K |S|^(n-1), clamped to [tau_min, tau_max] */
/* Explicit Smagorinsky: each node collides with the tau that the previous step stored for it and
 * stores tau0 + 3 Cs^2 |S| of the strain rate formed with that tau (a caller-owned tau field, see
 * lbm_bind_tau).  Its steady states are those of LBM_SMAG. */
#define LBM_SMAG_LAGGED 3
/* Smagorinsky on the traceless strain rate: tau = tau0 + 3 Cs^2 |S_d|, S_d = S - tr(S)/d I.  On
 * these moment bases S_d is proportional to s_nu, so tau is the larger root of a quadratic and is
 * computed in closed form (no sweeps).  Equal to LBM_SMAG when the flow has no bulk strain. */
#define LBM_SMAG_DEV 4

/* strain-rate routes */
#define LBM_YU 0
#define LBM_CHAI 1

/* boundary kinds per face */
#define LBM_PERIODIC 0
#define LBM_WALL 1
#define LBM_LID 2
/* Exchange face of a z-slab (both z faces of a 3D lattice, see lbm_halo_pack): the lattice is one
 * slab of a larger lattice cut along z, and its neighbouring slabs supply the populations that
 * enter through these faces.  The context then holds nz + 2 planes: plane 0 and plane nz + 1 are
 * ghost planes holding the neighbours' boundary populations, planes 1..nz are the slab's own.
 * Every buffer and field of the context spans all nz + 2 planes (N = nx ny (nz + 2)); steps,
 * read-outs and sums compute the own planes only; lbm_init fills the ghost planes with what the
 * first step pulls from them. */
#define LBM_HALO 3

/* Model parameters (plain data, copied by lbm_create).  |S| = sqrt(2 S:S).  With a closure, S
 * and tau are solved together at each node by fixed-point sweeps on tau from the same
 * pre-collision state: Smagorinsky takes exactly smag_iters sweeps from tau0; the power law
 * sweeps from tau0 until |tau_new - tau| <= pl_tol * tau_new or pl_max_iter sweeps. */
typedef struct lbm_params {
    int precision;   /* LBM_FP64, LBM_FP32, LBM_FP16S, LBM_BF16S */
    int closure;     /* LBM_NEWTON, LBM_SMAG, LBM_POWERLAW, LBM_SMAG_LAGGED, LBM_SMAG_DEV */
    int formula;     /* LBM_YU or LBM_CHAI: the route whose S feeds the closure in lbm_step */
    int smag_iters;  /* Smagorinsky sweeps, 1..64 (default 6) */
    int pl_max_iter; /* power-law sweep cap, 1..1000 (default 64) */
    int bc[6];       /* per face: LBM_PERIODIC, LBM_WALL or LBM_LID (default all periodic) */
    int force_field; /* 1: lbm_bind supplies a per-node force field; 0: the uniform force */
    double rho0;     /* mean density (default 1) */
    double smag_cs;  /* Smagorinsky constant Cs */
    double pl_n;     /* power-law index n > 0 */
    double pl_k;     /* power-law consistency K >= 0 */
    double pl_tau_min, pl_tau_max; /* clamp, 1/2 < tau_min <= tau_max (default 0.505, 5.0) */
    double pl_tol;   /* relative sweep tolerance (default 1e-13 for FP64, 1e-6 otherwise) */
    double lid_u[6][3]; /* wall velocity of each LBM_LID face */
} lbm_params;

typedef struct lbm_ctx lbm_ctx;

/* Fill *p with the defaults named above (FP32, Newtonian, Yu, all faces periodic, rho0 = 1).
 * p must not be NULL. */
void lbm_default_params(lbm_params* p);

/* Create a context for an nx x ny x nz lattice (nz = 1 for D2Q9).
 *  lattice  LBM_D2Q9, LBM_D3Q15 or LBM_D3Q19 (D2Q9: FP64 and FP32 storage only).
 *  rates    q relaxation rates s_0..s_{q-1} of the diagonal collision matrix, eq. (sD3Q15):
 *           the conserved entries (0, 3, 5, 7 in D3Q19 and D3Q15; 0, 3, 5 in D2Q9) must be 0,
 *           every other entry lies in (0, 2).  The viscous entries (9, 11, 13, 14, 15 in D3Q19;
 *           9..13 in D3Q15; 7, 8 in D2Q9) hold 1/tau0; they must be equal for the Yu route and
 *           for any closure.  On D2Q9 and D3Q15 the Yu route is the Yu-type formula that the
 *           Sec. 5.4 procedure derives from Chai's formula for that basis.
 *  force    d components of a uniform body-force density (rho0 g), or NULL for none.
 *  p        parameters, or NULL for the defaults.
 * Host pointers, read during the call only.  Errors: LBM_ERR_ARG for any violated rule above,
 * nx*ny*nz >= 2^31, or ny or nz > 65535; LBM_ERR_NOMEM / LBM_ERR_CUDA if the context's own
 * device scratch (a few KB of partial sums) cannot be allocated.  *out is set to NULL on error. */
int lbm_create(lbm_ctx** out, int lattice, int nx, int ny, int nz, const double* rates,
               const double* force, const lbm_params* p);

/* Free the context and the scratch it allocated.  Caller-owned buffers are untouched.
 * NULL is accepted. */
int lbm_destroy(lbm_ctx* ctx);

/* Population layout: the distribution functions f_i(x) of Sec. 2 (eq. (mrteq)) are stored as q
 * arrays of *stride elements of *elem_bytes bytes in each of the two buffers (stride >= N, a
 * multiple of 128).  Any output pointer may be NULL. */
int lbm_layout(const lbm_ctx* ctx, int* q, int64_t* stride, int* elem_bytes);

/* Bind caller-owned device memory for the populations of eq. (mrteq) and a CUDA stream
 * (cudaStream_t passed as void*, NULL = the legacy default stream).  f_a, f_b: q*stride elements each, 16-byte aligned, distinct.
 * force_field: d x N values of the compute type when the context was created with
 * p->force_field = 1 (must be non-NULL then), else ignored.  The buffers must stay valid until
 * the context is destroyed or re-bound.  After binding, A is the current buffer. */
int lbm_bind(lbm_ctx* ctx, void* f_a, void* f_b, const void* force_field, void* stream);

/* Bind the tau field of the LBM_SMAG_LAGGED closure: N values of the compute type (double for
 * LBM_FP64, float otherwise), caller-owned device memory, naturally aligned, valid until the
 * context is destroyed or re-bound.  lbm_init writes every node's first tau (the closure's value
 * at the prescribed gradient, tau0 without one); each lbm_step reads a node's entry and rewrites it
 * in place; read-outs read it.  The caller may read or overwrite it between calls (it is part of
 * the state: lbm_get_state / lbm_set_state do not copy it).  Other closures ignore it.  With the
 * lagged closure, lbm_init, lbm_step, lbm_strain_rate and lbm_macroscopic return LBM_ERR_STATE
 * until it is bound.  Errors: LBM_ERR_ARG for NULL or misaligned memory. */
int lbm_bind_tau(lbm_ctx* ctx, void* tau_field);

/* Initialise the current buffer so that the next step sees the pre-collision state
 *   f(x) = f_eq(drho, rho0 u) + T^-1 m_neq - Fbar/2,
 * where m_neq holds the first-order viscous non-equilibrium moments of the velocity gradient
 * given by eq. (YuLuobasis) of Sec. 4.1 (zero when grad_u is NULL) and Fbar is the discrete force.
 * drho (N), u (d x N), grad_u (d*d x N, entry a*d + b = du_a/dx_b): device pointers to double.
 * With a closure, s_nu in m_neq is the closure's value at the given gradient. */
int lbm_init(lbm_ctx* ctx, const double* drho, const double* u, const double* grad_u);

/* Advance n >= 0 time steps of the MRT lattice Boltzmann equation, eq. (mrteq) in its moment form
 * eq. (mrteqvT) (Sec. 2): each step pulls f_i(x) = f*_i(x - c_i) from the current buffer, relaxes
 * m - m_eq (eq. (meq)) with the diagonal rates of eq. (sD3Q15) at every node, the viscous rates
 * set by the closure from S of eq. (LuoS) or eq. (ChaiS) (p->formula), adds the discrete force,
 * and writes f* to the other buffer, which becomes current.
 * n = 0 does nothing.  Asynchronous on the bound stream.  The result does not depend on the
 * schedule (lbm_set_schedule): each node's arithmetic is the same whether the steps are launched
 * one at a time or several per launch.  A multi-step launch orders its tiles through
 * library-owned counters with bounded waits; a wait that runs out (none does while the launch
 * has the GPU to itself) is reported by the next lbm_sums or lbm_status as LBM_ERR_STATE. */
int lbm_step(lbm_ctx* ctx, int n);

/* How lbm_step(n >= 2) launches its steps.
 *  LBM_SCHEDULE_AUTO      several steps per launch when the storage is FP32/FP16S/BF16S, the
 *                         lattice is 3D with at most 2^22 nodes and
 *                         more units (a z plane times a band of y rows of about 1024-4096 nodes)
 *                         than the GPU holds resident blocks; one launch per step otherwise (the
 *                         default).  On larger lattices, and on D2Q9 lattices, a step boundary
 *                         costs less than the multi-step launch's synchronisation.
 *  LBM_SCHEDULE_PER_STEP  one launch per step.
 *  LBM_SCHEDULE_STREAM    several steps per launch wherever the storage allows it (not FP64),
 *                         whatever the lattice size.
 *  LBM_SCHEDULE_STALL_CHECK  diagnostic of the bounded waits, one-shot: the next lbm_step(n >= 2)
 *                         that can run several steps per launch starts that launch one step
 *                         ahead, so that every dependency wait runs out (about two seconds);
 *                         the launch ends, lbm_status then reports LBM_ERR_STATE, the state is
 *                         invalid and the schedule is back to LBM_SCHEDULE_AUTO.
 * A launch of several steps (at most 4096; lbm_step(n) makes as many launches as it needs) cuts
 * the lattice into units (one z plane by a band of y rows, all of x); a unit runs step k once its
 * neighbouring units (z +-1, band +-1, periodically wrapped) have completed step k-1, so
 * consecutive steps overlap instead of draining the GPU between them.
 * Errors: LBM_ERR_ARG for an unknown schedule. */
#define LBM_SCHEDULE_AUTO 0
#define LBM_SCHEDULE_PER_STEP 1
#define LBM_SCHEDULE_STREAM 2
#define LBM_SCHEDULE_STALL_CHECK 3
int lbm_set_schedule(lbm_ctx* ctx, int schedule);

/* Counters since lbm_create: *steps = time steps advanced by lbm_step, *step_launches = step
 * kernels it launched for them (one per step, or one per multi-step launch).  Either pointer may
 * be NULL.  Host-side; no synchronisation. */
int lbm_stats(const lbm_ctx* ctx, int64_t* steps, int64_t* step_launches);

/* Failure detector: a watchdog on the conservation laws of the scheme.  With every >= 1, each
 * lbm_step(n) advances in chunks of at most `every` steps and after each chunk computes the
 * global sums of lbm_sums (synchronising the bound stream) and checks them against reference
 * sums, taken from the state at the first lbm_step after lbm_set_watchdog, lbm_bind, lbm_init,
 * lbm_set_state or lbm_adjoint:
 *  - every sum finite, else LBM_ERR_NONFINITE;
 *  - the total mass sum delta rho equal to the reference (the collision conserves mass, eq.
 *    (mrteqvT) with s_0 = 0, and so do the periodic, wall and moving-wall rules), else
 *    LBM_ERR_DRIFT;
 *  - on a lattice with every face periodic and no per-node force field, each total momentum
 *    component equal to the reference plus k N F after k steps (the collision conserves j,
 *    s_3 = s_5 = s_7 = 0, and the force adds F per node and step), else LBM_ERR_DRIFT.
 * Each bound is tol * N * rho0 (absolute, in the units of the sums).  On a failure lbm_step
 * returns at once; the state is the one after the chunk that failed, the steps run so far are
 * counted by lbm_stats, and lbm_last_error names the quantity, its deviation and the bound.
 * every = 0 (the default) turns the watchdog off; with it on, lbm_step is synchronous and the
 * chunking costs one extra read of the populations per chunk (results are unchanged: they do
 * not depend on how the steps are split into launches).
 * Errors: LBM_ERR_ARG for every < 0, or a negative or non-finite tol when every > 0. */
int lbm_set_watchdog(lbm_ctx* ctx, int every, double tol);

/* Synchronise the bound stream and report the library's asynchronous status: LBM_ERR_CUDA for a
 * failed kernel, LBM_ERR_STATE (once; the record is then cleared) when a multi-step launch
 * stopped because a wait for neighbouring units ran out, LBM_OK otherwise (also when nothing is
 * bound). */
int lbm_status(lbm_ctx* ctx);

/* Strain rate S_ab = (d_a u_b + d_b u_a)/2 of the state the next step sees (Sec. 3), by
 * `formula`: LBM_YU, eq. (LuoS) (on D2Q9 and D3Q15 the Yu-type formula of the Sec. 5.4
 * procedure), or LBM_CHAI, eq. (ChaiS); with the closure solved as in a step.  S_out: ns x N values of the compute type (ns = 6 in 3D, 3 in
 * 2D); tau_out: N values or NULL.  Device pointers.  LBM_YU requires equal viscous rates. */
int lbm_strain_rate(lbm_ctx* ctx, int formula, void* S_out, void* tau_out);

/* Macroscopic fields of the state the next step sees, as Sec. 2 defines them for the
 * delta-rho form of eq. (edf): drho = sum f (N values) and u = j/rho0, j = sum c f + F/2 (the
 * force half-shift of the discrete force) (d x N values), compute type, device pointers (either
 * may be NULL). */
int lbm_macroscopic(lbm_ctx* ctx, void* drho_out, void* u_out);

/* Global sums of the state the next step sees, accumulated in FP64 on the device, of the Sec. 2
 * conserved moments (delta rho and j of eq. (moment)): out[0] = sum delta rho, out[1..d] = sum j
 * (j = sum c f + F/2).  out is a HOST pointer to d+1
 * doubles.  Synchronises the bound stream.  Returns LBM_ERR_NONFINITE (with out filled) if a sum
 * is NaN or infinite, LBM_ERR_STATE as lbm_status does. */
int lbm_sums(lbm_ctx* ctx, double* out);

/* Copy the current buffer's populations (the state f of eq. (mrteq); checkpoint and restart) to
 * dst / from src as a dense q x N array of the storage type (no stride padding).  dst/src may be host or device memory (pinned host memory gives
 * asynchronous copies; pageable host memory makes the call synchronous). */
int lbm_get_state(lbm_ctx* ctx, void* dst);
int lbm_set_state(lbm_ctx* ctx, const void* src);

/* Allocation-free global sums (the paper has no counterpart: this is a library service).
 *
 * The same sums as lbm_sums, equal to rounding (the rows are split among blocks differently, so
 * the additions run in another order), for callers that cannot allocate device memory at the
 * point where they need the sums: lbm_create allocates the context's scratch with cudaMalloc, which such
 * callers must avoid, e.g. code whose device memory belongs to another allocator (a framework's
 * caching pool) or a time-stepping loop with a latency budget (cudaMalloc / cudaFree may
 * synchronise the device and take unbounded time).  No context is used and nothing is allocated:
 * no cudaMalloc, cudaFree or allocating library routine is called.
 *  lattice, nx, ny, nz  as for lbm_create (16-bit storage: D3Q19 and D3Q15);  p: precision, bc,
 *           lid_u and rho0 are read;
 *  force    d components of the uniform force density, or NULL;
 *  f        device pointer to one population buffer (q arrays of `stride` elements of the
 *           storage type, stride >= nx*ny*nz), holding post-collision populations as after
 *           lbm_step; the sums are those of the state the next step would see;
 *  force_field  d x N values of the compute type, or NULL (then `force` applies);
 *  out      HOST pointer to d+1 doubles: [sum delta rho, sum j_x, sum j_y, (sum j_z)];
 *  stream   cudaStream_t as void* (NULL = legacy default stream); the call synchronises it.
 * The scratch is one static device array of LBM_NOALLOC_MAX_BLOCKS x 4 partial sums (plus 4
 * doubles) that every GPU loading the library holds until the process exits.  Lattices with
 * more than LBM_NOALLOC_MAX_ROWS rows (ny * nz) are rejected with LBM_ERR_ARG, as are the
 * argument errors of lbm_create that apply here (dimensions, precision, rho0 > 0 and finite,
 * finite force and wall velocities, boundary pairs); a rejected call touches no CUDA state.
 * Every call looks up the array's device address on the current device (cudaGetSymbolAddress,
 * which allocates nothing), so the call stays valid after a device reset.  The call synchronises
 * its stream, so it must not be called while that stream is being captured into a CUDA graph.
 * Each call writes every scratch slot it reads,
 * so nothing has to be cleared between calls, but all calls share the one array: calls whose
 * kernels can overlap on the GPU (other streams or host threads) race and must be serialised.
 * Returns LBM_OK, LBM_ERR_ARG, LBM_ERR_CUDA, or LBM_ERR_NONFINITE (out filled) for a NaN or
 * infinite sum. */
#define LBM_NOALLOC_MAX_BLOCKS 16384
#define LBM_NOALLOC_MAX_ROWS (16 * LBM_NOALLOC_MAX_BLOCKS)
int lbm_sums_noalloc(int lattice, int nx, int ny, int nz, const lbm_params* p, const double* force,
                     const void* f, int64_t stride, const void* force_field, double* out, void* stream);

/* Gradient of the dissipation functional with respect to the body-force field (adjoint).
 *
 *   L(g) = sum_x nu_eff(x) sum_ab S_ab(x)^2,   nu_eff = (tau - 1/2)/3,
 * with S and tau (closure included) of the pre-collision state that step T+1 would see, after
 * T steps from the current state under the bound force field F = rho0 g.  dL/dg comes from a
 * hand-written reverse pass of the full step (Yu-form strain rate, which equals Chai's, Sec. 5.1;
 * the closure differentiated at its converged fixed point; |S| = 0 contributes no closure term),
 * with sqrt(T)-style checkpointing: every seg-th state is kept during the forward pass and each
 * segment is recomputed from its checkpoint during the reverse sweep (about 2T forward steps and
 * T reverse steps in all).  The force gradient accumulates in the compute type within a segment
 * and in FP64 across segments.
 * Supported: D3Q19, LBM_FP32 or LBM_FP64 populations, LBM_NEWTON or LBM_SMAG, all faces
 * periodic, a force field bound (p->force_field = 1); otherwise LBM_ERR_ARG.
 *  work     caller-owned device workspace of at least lbm_adjoint_workspace() bytes, 256-byte
 *           aligned (checkpoints, segment states, two adjoint buffers, accumulators);
 *  dLdg     device pointer to 3 x N doubles, overwritten with dL/dg (component-major);
 *  loss     HOST pointer to one double, set to L.
 * After the call the current buffer holds the state after T steps.  Synchronises the stream. */
int lbm_adjoint_workspace(lbm_ctx* ctx, int T, int seg, int64_t* bytes);
int lbm_adjoint(lbm_ctx* ctx, int T, int seg, void* work, int64_t work_bytes, double* dLdg, double* loss);

/* Domain decomposition along z (the lattice is cut into slabs of whole z planes, one per context
 * and usually one per GPU; the paper's method is local in space, Sec. 1 notes the natural
 * parallelism of the lattice Boltzmann equation).  A context created with bc[4] = bc[5] =
 * LBM_HALO steps its own planes; between two steps the populations that cross each z face move
 * to the neighbouring slab:
 *   lbm_halo_pack    copies, from the current buffer, the post-collision populations with c_z = +1
 *                    of the top own plane (z = nz) into send_hi and those with c_z = -1 of the
 *                    bottom own plane (z = 1) into send_lo;
 *   lbm_halo_unpack  writes recv_lo (the lower neighbour's send_hi) into the populations with
 *                    c_z = +1 of ghost plane 0 and recv_hi (the upper neighbour's send_lo) into the
 *                    populations with c_z = -1 of ghost plane nz + 1.
 * Each halo buffer holds `pops` arrays of nx * ny elements of the storage type (population order:
 * increasing index among those crossing the face; 5 for D3Q19 and D3Q15), device memory,
 * caller-owned, `elems` = pops * nx * ny (lbm_halo_layout).  Slab k's upper neighbour is slab
 * k + 1 (periodically: the lattice as a whole is periodic in z); one slab is its own neighbour.
 * Stepping then goes step(1), pack, exchange (the caller's: NCCL send/recv between GPUs, or a
 * copy), unpack, step(1), ...; after lbm_init the ghost planes already hold what the first step
 * pulls.  With halo faces lbm_step takes n <= 1 (the exchange sits between steps), the watchdog and
 * the adjoint are not available (LBM_ERR_ARG), and lbm_sums sums the own planes (the lattice's
 * totals are the sums over the slabs).  Asynchronous on the bound stream.
 * Errors: LBM_ERR_ARG for a context without halo faces or NULL buffers. */
int lbm_halo_layout(const lbm_ctx* ctx, int* pops, int64_t* elems);
int lbm_halo_pack(lbm_ctx* ctx, void* send_lo, void* send_hi);
int lbm_halo_unpack(lbm_ctx* ctx, const void* recv_lo, const void* recv_hi);

/* Message of the last failed call on ctx (empty if none), owned by the context.  With ctx = NULL:
 * the message of the last failed lbm_create on the calling thread. */
const char* lbm_last_error(const lbm_ctx* ctx);

#ifdef __cplusplus
}
#endif

#endif /* LBM_H */
