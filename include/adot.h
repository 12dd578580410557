/*
 * adot.h - C ABI of the GB300 (sm_103a) A-DOT library.
 *
 * A-DOT is the Dumbser-Osher-Toro (DOT) path-conservative scheme for the 1D
 * de Saint Venant-Exner system with the flux-matrix eigenstructure computed
 * analytically (Carraro, Valiani & Caleffi, arXiv 1912.04791, Sec. 3.3).
 * The state is W = [h, q, z] (depth, unit discharge, bed elevation) on n
 * uniform cells of [x_min, x_max]; Eq. scheme (S = 0) advances it by
 *     W_i <- W_i - dt/dx (D-_{i+1/2} + D+_{i-1/2}),
 * with the DOT fluctuations of Eq. DOTjumpN (3-point Gauss-Legendre rule on
 * the segment path of Eq. path) and |A| = R|Lambda|R^-1 (Eq. asbA) from the
 * trigonometric roots of Eq. lambda and the vectors of Eq. RR / RR-1.
 *
 * Conventions for every entry point:
 *  - Pointers are plain host or device addresses; arrays are float64.
 *    A [3][n] array holds row 0 = h, row 1 = q, row 2 = z, each contiguous.
 *  - `on_device` = 1: the pointers are device addresses on the context's
 *    device (e.g. torch CUDA tensors' data_ptr()); 0: host addresses. The
 *    library copies in and out; it never keeps a caller pointer after the call.
 *  - The library allocates and owns all device state (state buffers, control
 *    block, scratch, CUDA graphs) from adot_create until adot_destroy.
 *  - Every call returns an adot_status and never throws. A device-side error
 *    (non-finite value, h <= 0, non-hyperbolic state) is recorded in a sticky
 *    device status word and returned by the next synchronising call; the
 *    context stays valid so that adot_get_state can still read the state.
 *  - Work is ordered on the CUDA stream given at creation (NULL: a stream the
 *    library creates). A context is not thread-safe. The warp-tile step
 *    kernels are launched with programmatic dependent launch: each may be
 *    scheduled while the kernel before it on the stream drains, but it reads
 *    nothing until that kernel has completed, so work the caller puts on the
 *    same stream is ordered as with ordinary launches.
 *  - There is no CPU fallback: without a usable CUDA device adot_create fails
 *    with ADOT_E_CUDA.
 */
#ifndef ADOT_H
#define ADOT_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
  ADOT_OK = 0,
  ADOT_E_INVALID_ARG = 1,       /* bad pointer, size, config value or call order */
  ADOT_E_NONPOSITIVE_DEPTH = 2, /* a cell reached h <= 0 */
  ADOT_E_NONFINITE = 3,         /* NaN or Inf in the state or the time step */
  ADOT_E_NONHYPERBOLIC = 4,     /* |k2 / sqrt(4 k1^3)| > 1 + 1e-6 at some state (Eq. parameters) */
  ADOT_E_CUDA = 5,              /* a CUDA runtime call failed */
  ADOT_E_TIMEOUT = 6,           /* a bounded device-side wait ran out */
  ADOT_E_UNSUPPORTED = 7        /* valid request this build does not implement */
} adot_status;

/* Sediment transport closure (Sec. 2). */
typedef enum {
  ADOT_LAW_GRASS = 0, /* q_s = A_g u^3 (Eq. Grass) */
  ADOT_LAW_MPM = 1,   /* q_s = sign(u) 8 (theta-0.047)_+^1.5 sqrt(g (s-1) d50^3), Eq. MPM,
                         theta = n^2 u^2 / ((s-1) d50 h^(1/3)) (Eq. Shields, Manning s_f) */
  ADOT_LAW_GRASS_THR = 2, /* q_s = A_g (u - u_cr)^3 (Eq. GrassThr), read as
                             A_g sign(u) max(|u| - u_cr, 0)^3: no transport at or below u_cr */
  ADOT_LAW_POWER = 3      /* q_s = A_g sign(u) max(|u| - u_cr, 0)^beta, beta >= 1: the power
                             law of Eq. Soni_qs (alpha = A_g, u_cr = 0); beta = 3 is
                             ADOT_LAW_GRASS_THR */
} adot_law_kind;

/* Arithmetic of the state and the fluctuations. */
typedef enum {
  ADOT_FP64 = 0, /* everything in float64 */
  ADOT_FP32 = 1  /* state as float-float (two float32 per value, updated with TwoSum);
                    fluctuations in float32; an edge with a quadrature node where
                    1 - arg^2 < 1e-4 (near-coalescent roots) redone in float64 */
} adot_precision;

/* Jump function of Eq. scheme. */
typedef enum {
  ADOT_SCHEME_DOT = 0,    /* DOT fluctuations (Eq. DOTjumpN) with the analytic eigenstructure
                             (A-DOT, Sec. 3.3) */
  ADOT_SCHEME_PRICE_C = 1 /* PRICE-C, the paper's centred comparison scheme (Sec. 3.2):
                             D-/+ = 1/4 [2 A^Psi -/+ (dx/dt) I_eps -/+ (dt/dx) (A^Psi)^2] dW
                             (Eq. PRICEjump, AiPRICE), A^Psi the 3-point Gauss-Legendre mean
                             of A along the segment path (Eq. Apsi), I_eps = diag(1, 1, eps)
                             acting on (h, q, z) (Eq. Im); dt from the same CFL rule */
} adot_scheme;

/* Boundary kinds. A ghost cell outside each end supplies the edge state. */
typedef enum {
  ADOT_BC_TRANSMISSIVE = 0, /* ghost = adjacent cell (zero jump, zero fluctuation) */
  ADOT_BC_PERIODIC = 1,     /* both ends: the domain wraps */
  ADOT_BC_INFLOW_Q = 2,     /* ghost q = value[0]; h, z copied */
  ADOT_BC_OUTFLOW_H = 3,    /* ghost h = value[0]; q, z copied */
  ADOT_BC_INFLOW_QZ = 4,    /* ghost q = value[0], z = value[1] - value[2] * t; h copied */
  ADOT_BC_INFLOW_QS = 5,    /* sediment feed (Sec. 5.1): ghost q = value[0], h copied, z
                               continued linearly from the two cells next to the end
                               (2 z_1 - z_2); the bed discharge through the end edge is
                               xi * value[1] exactly (value[1] = q_s,in, signed along +x):
                               the edge's bed fluctuation on the cell side becomes
                               xi (q_s(W_cell) - q_s,in) at the left end and
                               xi (q_s,in - q_s(W_cell)) at the right end */
  ADOT_BC_OUTFLOW_HS = 6    /* ghost h = value[0], q copied, z continued linearly */
} adot_bc;

typedef struct {
  int32_t kind;     /* adot_law_kind */
  double g;         /* gravitational acceleration [m/s^2] */
  double xi;        /* 1 / (1 - p), p = bed porosity (Eq. SV-Ex3) */
  double Ag;        /* Grass coefficient [s^2/m] */
  double s_rel;     /* MPM: relative grain density */
  double d50;       /* MPM: median grain size [m] */
  double manning_n; /* MPM: Manning coefficient [s/m^(1/3)] */
  double u_cr;      /* Grass with threshold / power law: incipient velocity [m/s], >= 0 */
  double beta;      /* power law: exponent, >= 1 (ignored by the other kinds) */
} adot_law;

typedef struct {
  int64_t n_cells;          /* >= 1 */
  double x_min, x_max;      /* domain, x_max > x_min */
  double cfl;               /* dt = cfl * dx / max_i max(|l1|, |l3|)(W_i), 0 < cfl <= 1 */
  adot_law law;
  int32_t precision;        /* adot_precision */
  int32_t bc_left, bc_right;
  double bc_left_value[3], bc_right_value[3];
  int32_t block_threads;    /* threads per block of the step kernel: 128, 256, 512; 0 = autotuned */
  int32_t steps_per_graph;  /* time steps captured per CUDA graph; 0 = default (48) */
  int32_t device;           /* CUDA device ordinal; -1 = the calling thread's current device */
  int32_t reg_cap;          /* register cap per thread of the step kernel: 64 (block kernel
                               or warp tiles), 72 (warp tiles, 128 threads), 80 (warp tiles,
                               256 threads), 40 or 32 (warp tiles, 256 threads, PRICE-C only),
                               or -1 = none (block kernel); 0 = autotuned */
  int32_t step_kernel;      /* 1 = block kernel (B-1 cells per block, shared-memory exchange),
                               2 = persistent warps, each over a contiguous range of cells
                               in chunks of 32 edges (shuffle exchange); 0 = autotuned */
  double ks;                /* Strickler coefficient K_s [m^(1/3)/s] of the friction source
                               S = (0, -g h s_f, 0), s_f = q|q| / (K_s^2 h^(10/3)) (Sec. 2),
                               added as dt S(W_i^n) in Eq. scheme; 0 = frictionless */
  int32_t order;            /* 0 or 1: the first-order scheme (Eq. scheme); 2: second-order
                               MUSCL-Hancock variant (minmod slopes of h + z, q, z, Hancock
                               half-step predictor, DOT edges between the predicted states
                               plus the path integral of A inside each cell; Sec. 6 leaves
                               the order open). Order 2 runs the warp-tile kernel only
                               (step_kernel 0 or 2) and is frictionless without a feed
                               (ks = 0, no ADOT_BC_INFLOW_QS): ADOT_E_UNSUPPORTED otherwise */
  int32_t scheme;           /* adot_scheme; 0 = DOT. PRICE-C runs the first-order warp-tile
                               kernel of 256 threads (register cap 64, 40 or 32; 0 = autotuned):
                               order 2, step_kernel 1 and other shapes give ADOT_E_UNSUPPORTED;
                               it takes the friction source and the boundary kinds as DOT does */
  double price_eps;         /* PRICE-C: epsilon of I_eps (Eq. Im), >= 0 (the paper's Tests 1
                               and 2 use 1e-4); ignored by DOT */
} adot_config;

typedef struct adot_ctx adot_ctx;

/* Creates a context: validates cfg (ADOT_E_INVALID_ARG on a bad value; both ends
 * must be periodic or neither), makes cfg->device current (unless -1), allocates
 * the device state and control block on it and binds `cuda_stream` (a cudaStream_t, or NULL). The
 * state is zero until adot_set_state. *out receives the context or NULL. */
adot_status adot_create(const adot_config* cfg, void* cuda_stream, adot_ctx** out);

/* Frees everything the context owns. Accepts NULL. */
void adot_destroy(adot_ctx* ctx);

/* Copies the state in (n_cells float64 values each), resets time to t0 and the
 * step counter to 0, and computes the first time step's CFL maximum.
 * ADOT_E_NONPOSITIVE_DEPTH / ADOT_E_NONFINITE if the state is not admissible. */
adot_status adot_set_state(adot_ctx* ctx, const double* h, const double* q, const double* z,
                           int on_device, double t0);

/* Copies the current state out (float-float states are summed to float64). */
adot_status adot_get_state(adot_ctx* ctx, double* h, double* q, double* z, int on_device);

/* Checkpoint and resume. A checkpoint is one byte blob: a 128-byte header
 * (magic "ADOT", version 1, n_cells, precision, law, time, last dt, step
 * count, the spectral-radius maximum the next step's dt is taken from, the
 * sticky device status, and a 64-bit FNV-1a fingerprint of the config fields
 * that enter the arithmetic: n_cells, domain, cfl, law, precision and both
 * boundary conditions; not the launch shape), followed by the state's stored
 * words as rows h, q, z of n 8-byte values each (float64 in ADOT_FP64, the
 * (hi, lo) float32 pair of the float-float value in ADOT_FP32: nothing is
 * rounded). Restoring it into a context of the same config makes every later
 * step bit-identical to the steps the saved context would have taken.
 *
 * adot_checkpoint_size: *bytes_out = 128 + 24 n.
 * adot_checkpoint_save: writes the blob to `buf` (host, or device when
 *   on_device = 1) of `bytes` >= that size; ADOT_E_INVALID_ARG before a state
 *   was set or when the buffer is short. Waits for the stream.
 * adot_checkpoint_load: reads a blob; ADOT_E_INVALID_ARG when the magic, the
 *   version, the sizes or the fingerprint do not match this context (the state
 *   is then left as it was). Resets the step-phase bookkeeping as
 *   adot_set_state does, but keeps the saved time and step count; returns the
 *   saved sticky status, if any. */
adot_status adot_checkpoint_size(adot_ctx* ctx, int64_t* bytes_out);
adot_status adot_checkpoint_save(adot_ctx* ctx, void* buf, int64_t bytes, int on_device);
adot_status adot_checkpoint_load(adot_ctx* ctx, const void* buf, int64_t bytes, int on_device);

/* Advances n_steps >= 0 time steps (Eq. scheme) with no end time, then waits
 * for the stream and reports the time and the last step's dt (either pointer
 * may be NULL) and the first device-side error. */
adot_status adot_step(adot_ctx* ctx, int64_t n_steps, double* t_out, double* dt_last_out);

/* Enqueues n_steps steps on the stream and returns without waiting (errors
 * surface at the next synchronising call: adot_step, adot_run_to, adot_query). */
adot_status adot_enqueue_steps(adot_ctx* ctx, int64_t n_steps);

/* Advances until the time reaches t_end (the last step is shortened to land on
 * it exactly). *steps_out (may be NULL) receives the steps taken by this call. */
adot_status adot_run_to(adot_ctx* ctx, double t_end, int64_t* steps_out);

/* Waits for the stream; reports time, total steps since adot_set_state and the
 * last dt (NULL pointers are skipped) and the first device-side error. */
adot_status adot_query(adot_ctx* ctx, double* t_out, int64_t* steps_out, double* dt_last_out);

/* DOT fluctuations of n independent edges (Eq. DOTjumpN, G = 3, segment path),
 * in the context's law and precision (also in a PRICE-C context). WL, WR: [3][n] left and right states;
 * Dminus, Dplus: [3][n] outputs. rho_max_out (may be NULL): the largest
 * max(|l1|, |l3|) met at any quadrature node. n = 0 is valid and writes nothing.
 * In ADOT_FP32 the inputs are first rounded to float-float, as the state is. */
adot_status adot_fluctuations(adot_ctx* ctx, const double* WL, const double* WR, int64_t n,
                              double* Dminus, double* Dplus, double* rho_max_out,
                              int on_device);

/* PRICE-C fluctuations of n independent edges (Eq. PRICEjump, Eq. AiPRICE, G = 3
 * Gauss-Legendre nodes for A^Psi) with dt/dx = dt_over_dx > 0 and the context's
 * law, precision and price_eps (whatever the context's scheme). WL, WR, Dminus,
 * Dplus as for adot_fluctuations ([3][n] float64; in ADOT_FP32 the inputs are
 * first rounded to float-float). n = 0 is valid and writes nothing.
 * ADOT_E_INVALID_ARG for a non-positive or non-finite dt_over_dx. */
adot_status adot_price_fluctuations(adot_ctx* ctx, const double* WL, const double* WR, int64_t n,
                                    double dt_over_dx, double* Dminus, double* Dplus,
                                    int on_device);

/* Times the compiled step-kernel variants allowed by the configuration (kernel
 * kind, block size and register cap; a field left at 0 is free) on the current state with
 * `trial_steps` steps each, keeps the fastest and re-captures the time-loop
 * graph. Trial steps write only the scratch buffer, so the state and time do
 * not advance. The choice is cached per (device, law, precision, log2 n) for
 * the process; adot_set_state runs this once per context with trial_steps = 8
 * when a field is free and nothing is cached. block_out, reg_cap_out and
 * step_kernel_out (each may be NULL) receive the choice. ADOT_E_INVALID_ARG before adot_set_state. */
adot_status adot_autotune(adot_ctx* ctx, int64_t trial_steps, int32_t* block_out,
                          int32_t* reg_cap_out, int32_t* step_kernel_out);

/* Precision diagnostic of the current state (not a step): *nodes_out (may be
 * NULL) receives the quadrature nodes of one step, 3 per edge (edges 0..n, or
 * 0..n-1 when periodic); *fp64_nodes_out (may be NULL) how many of them fail
 * the float32 step kernels' test for nearly coalescing roots of Eq. lambda
 * (1 - arg^2 < 1e-4 with arg = k2 / sqrt(4 k1^3), Eq. parameters, or arg not
 * finite), by the same float32 test on the same node values, run in a
 * separate kernel; an edge with such a node is redone in float64 by the step.
 * ADOT_FP64 contexts report 0. Waits for the stream.
 * ADOT_E_INVALID_ARG before a state was set. */
adot_status adot_precision_stats(adot_ctx* ctx, int64_t* nodes_out, int64_t* fp64_nodes_out);

/* Sums over the cells of h, q and z (float64, fixed-order tree: the result is
 * bit-reproducible). Multiply by dx for the integrals. */
adot_status adot_conserved_sums(adot_ctx* ctx, double sums_out[3]);

/* ---- Batched ensembles of independent channels ------------------------------
 * Each channel is a separate dSVE problem advanced by Eq. scheme with the DOT
 * fluctuations of Eq. DOTjumpN and its own time step dt_c = cfl dx_c / rho_c
 * (reading of the unstated CFL rule as for a single channel), Grass law
 * (Eq. Grass) with a per-channel A_g, transmissive ends. The channels' cells lie
 * end to end in the state arrays: channel c owns cells off[c] .. off[c+1]-1 with
 * off[c] = n_cells[0] + ... + n_cells[c-1]. Channels stop at t_end individually.
 *
 * Two forms run the channels. Persistent channel loops: one launch per run_to
 * (per 16384 steps of the longest-running channel); each CTA takes whole
 * channels from a device queue, largest estimated work first (N_c^2 rho_c /
 * length_c for run_to, N_c for step), and steps each to t_end in a
 * device-side loop with one block barrier per step; no CTA waits on another,
 * so a channel longer than a CTA's share of the work sets the run time.
 * Per-step launches: one launch (captured in CUDA graphs) advances every
 * running channel by one of its own steps, over a tile list of all channels.
 * Both evaluate the same edges and cells. */
typedef struct {
  int32_t n_channels;       /* >= 1 */
  const int64_t* n_cells;   /* host [n_channels], each >= 1 */
  const double* length;     /* host [n_channels], channel length [m] (dx_c = length/n_cells) */
  const double* Ag;         /* host [n_channels], Grass coefficient [s^2/m] */
  double g, xi, cfl;        /* shared: gravity, 1/(1-p), CFL number in (0, 1] */
  int32_t precision;        /* ADOT_FP64 or ADOT_FP32 (float-float state) */
  int32_t block_threads;    /* threads per block. Persistent channel loops: 256, 384, 512
                               or 768 (0 = 384 or 768, the better balanced). Per-step: 128,
                               256, 512 (block kernel:
                               tile = block_threads - 1 cells; warp tiles: 256 only);
                               0 = autotuned */
  int32_t steps_per_graph;  /* per-step launches captured per CUDA graph; 0 = default (48) */
  int32_t device;           /* CUDA device ordinal; -1 = current */
  int32_t step_kernel;      /* 0 = chosen at each set_state (default): persistent channel loops
                               (one CTA per channel, or the long channels on cluster teams)
                               when the estimated list schedule of the channels onto the CTAs
                               is within 1/0.85 of balanced, else per-step launches (4);
                               3 = persistent channel loops, the better estimated plan;
                               5 = persistent with cluster teams (block_threads 0 or 768);
                               per-step launches: 1 = block kernel, 2 = persistent warp tiles
                               (31 cells per tile, shuffle exchange, no block barrier), 4 = the
                               faster of 1 and 2 by trial launches */
} adot_ensemble_config;

typedef struct adot_ensemble adot_ensemble;

/* Creates an ensemble: validates cfg (ADOT_E_INVALID_ARG), copies the host
 * arrays, allocates the device state (two ping-pong copies of all cells), the
 * per-channel control arrays and the tile list (channels longest first). */
adot_status adot_ensemble_create(const adot_ensemble_config* cfg, void* cuda_stream,
                                 adot_ensemble** out);
void adot_ensemble_destroy(adot_ensemble* ens);

/* Copies in the concatenated float64 state (sum n_cells values each, host or
 * device per on_device), puts every channel at t = 0 with no steps taken and
 * computes each channel's first CFL maximum (persistent form: and orders the
 * channel queue by estimated work). Per-step form with block_threads = 0: the
 * first call times the tile sizes (two trial launches each, state unchanged). */
adot_status adot_ensemble_set_state(adot_ensemble* ens, const double* h, const double* q,
                                    const double* z, int on_device);
adot_status adot_ensemble_get_state(adot_ensemble* ens, double* h, double* q, double* z,
                                    int on_device);

/* Advances every channel until its own time reaches t_end (last step shortened
 * to land on it). *launches_out (may be NULL): step-kernel launches issued. The
 * persistent form continues channels that reached an earlier t_end; the
 * per-step form leaves a channel frozen once it has reached one (until the next
 * set_state). A non-finite value or non-positive depth ends the call with its
 * status (persistent form: every CTA stops after its current step). */
adot_status adot_ensemble_run_to(adot_ensemble* ens, double t_end, int64_t* launches_out);

/* Advances every channel by n_steps of its own steps (no end time). */
adot_status adot_ensemble_step(adot_ensemble* ens, int64_t n_steps);

/* Per-channel time and step count (host arrays [n_channels], may be NULL) and
 * the total cell-updates sum_c steps_c n_cells_c; waits for the stream. */
adot_status adot_ensemble_query(adot_ensemble* ens, double* t_out, int64_t* steps_out,
                                int64_t* cell_updates_out);

/* Variant in use: threads per block, number of tiles (persistent form: of
 * channels), the resident grid and the step kernel (1 block, 2 warp tiles,
 * 3 persistent channel loops); NULL pointers are skipped. */
adot_status adot_ensemble_info(adot_ensemble* ens, int32_t* block_out, int64_t* tiles_out,
                               int32_t* grid_out, int32_t* step_kernel_out);

/* The plan that run_to (which = 0) or step (which = 1) follows, chosen at the
 * last set_state (no counterpart in the paper). *form_out: 3 = persistent
 * channel loops, 1 or 2 = per-step launches (block / warp tiles);
 * *cluster_out: 1 = one CTA per channel, 2 or 4 = the long channels stepped by
 * teams of that many CTAs (a thread-block cluster; one exchange of the CFL
 * maximum through distributed shared memory per step), the others one CTA
 * each; *teamed_out: channels run by teams; *imbalance_out: the persistent
 * form's estimated list-scheduling makespan / mean CTA load. NULL pointers are
 * skipped. ADOT_E_INVALID_ARG for another `which`. */
adot_status adot_ensemble_plan(adot_ensemble* ens, int32_t which, int32_t* form_out, int32_t* block_out,
                               int32_t* cluster_out, int32_t* grid_out, int32_t* teamed_out,
                               double* imbalance_out);

/* Test hook of the cluster-team form's failure detection (no counterpart in
 * the paper). kind 1: in the next launch of the team form, CTA 1 of cluster 0
 * does not arrive at its first team exchange, so both members' bounded waits
 * (about 2^31 clock cycles, ~1 s) run out; the kernel records ST_TIMEOUT, every
 * CTA leaves, and run_to / step return ADOT_E_TIMEOUT with the context usable
 * (set_state starts over). kind 0 clears it. Nothing faults or hangs.
 * ADOT_E_INVALID_ARG for another kind. */
adot_status adot_ensemble_inject_fault(adot_ensemble* ens, int32_t kind);

/* ---- Learned surrogate of the quadrature-averaged |A| ----------------------
 * |A|_Psi = sum_k w_k |A(Psi(s_k))|, the matrix that multiplies W+ - W- in the
 * dissipative half of Eq. DOTjumpN, is approximated by a multilayer perceptron
 * 7 -> 128 -> 128 -> 128 -> 128 -> 9 with GELU hidden activations (tanh form),
 * bfloat16 weights and activations and float32 accumulation on tensor cores.
 * Inputs: standardised (h_L, q_L, z_L, h_R, q_R, z_R, A_g); outputs: the
 * standardised 9 entries of |A|_Psi (row-major). Training minimises the mean
 * squared error with Adam (beta1 0.9, beta2 0.999, eps 1e-8, cosine-decayed
 * step size to 5% of lr). Parameters are exchanged as one float32 vector, layer
 * by layer, W_l ([out][in] row-major) then b_l: 51721 values. */
typedef struct adot_mlp adot_mlp;
#define ADOT_MLP_PARAMS 51721

/* Allocates a network (parameters zero) for batches up to max_batch rows. */
adot_status adot_mlp_create(int64_t max_batch, void* cuda_stream, adot_mlp** out);
void adot_mlp_destroy(adot_mlp* mlp);
/* Parameters in (host [ADOT_MLP_PARAMS]); resets the Adam moments and step. */
adot_status adot_mlp_set_params(adot_mlp* mlp, const float* params);
adot_status adot_mlp_get_params(adot_mlp* mlp, float* params);
/* Engine of the surrogate step's fused inference: 0 = tcgen05, warp-specialised
 * three-tile pipeline (default); 1 = mma.sync; 2 = tcgen05, two independent
 * tile groups per CTA. ADOT_E_INVALID_ARG for another value. */
adot_status adot_mlp_set_engine(adot_mlp* mlp, int engine);
/* Engine of the training kernels (adot_mlp_train, adot_mlp_gradient and
 * adot_mlp_forward with fused = 0): 0 = tcgen05.mma with tensor-memory
 * accumulators (default): the forward pass in the fused two-group kernel
 * (fused = 2), which also stores every hidden layer's pre-activation and
 * activation, the backward layer products in 128-row x 64-column units, the
 * weight gradients with the batch rows as the reduction dimension; 1 =
 * mma.sync, one kernel per layer over 64-row tiles, GELU through tanhf. Both
 * take bf16 operands and accumulate in float32. ADOT_E_INVALID_ARG for another
 * value. A bounded device-side wait that runs out makes the call that launched
 * it return ADOT_E_TIMEOUT. */
adot_status adot_mlp_set_train_engine(adot_mlp* mlp, int engine);
/* Test hook for the failure detection of the tensor-core pipeline (no
 * counterpart in the paper): kind = 1 makes the next adot_mlp_forward with
 * fused = 3 withhold one accumulator hand-off in its first CTA, so that the
 * epilogue's bounded device-side wait (about 2^31 clock cycles, ~1 s) runs
 * out; that call returns ADOT_E_TIMEOUT and the network stays usable. The hook
 * clears itself after that one call; kind = 0 clears it. Nothing faults, traps
 * or hangs: every wait of the kernel is bounded and the products in flight
 * complete before its tensor memory is freed. */
adot_status adot_mlp_inject_fault(adot_mlp* mlp, int kind);
/* Training set: raw inputs X [n][7] and labels T [n][9] (float32, host or
 * device). Sets the standardisation (per-column mean and standard deviation)
 * and the training box (per-input min/max widened by 5% of the range). */
adot_status adot_mlp_set_data(adot_mlp* mlp, const float* X, const float* T, int64_t n,
                              int on_device);
/* stats32 (may be NULL): x mean[7], x sd[7], y mean[9], y sd[9]; box14 (may be
 * NULL): input lower bounds[7], upper bounds[7]. */
adot_status adot_mlp_get_stats(adot_mlp* mlp, float* stats32, float* box14);
/* Forward pass of n <= max_batch standardised inputs Xs [n][7] (host) to
 * standardised outputs Y [n][9] (host). fused = 0: the per-layer training
 * kernels (engine of adot_mlp_set_train_engine); 1: the single-kernel inference on mma.sync with the
 * tanhf GELU; 2 and 3: the single-kernel inference on the 5th-generation
 * tensor cores (tcgen05.mma, accumulators in tensor memory) with the
 * tanh.approx GELU, as two independent tile groups per CTA (2) or as the
 * warp-specialised three-tile pipeline (3) that the surrogate step uses by
 * default. ADOT_E_TIMEOUT if a bounded device-side wait for the tensor cores
 * ran out. */
adot_status adot_mlp_forward(adot_mlp* mlp, const float* Xs, int64_t n, float* Y, int fused);
/* Loss and gradient (host [ADOT_MLP_PARAMS]) of the mean squared error on a
 * batch of standardised inputs Xs [n][7] and targets Ts [n][9] (host). */
adot_status adot_mlp_gradient(adot_mlp* mlp, const float* Xs, const float* Ts, int64_t n,
                              float* loss_out, float* grad);
/* `steps` Adam steps on batches of `batch` rows drawn from the training set with
 * splitmix64(seed, step, row); loss_hist (host [steps], may be NULL) receives
 * each step's batch loss. One step is a replayed CUDA graph. */
adot_status adot_mlp_train(adot_mlp* mlp, int64_t steps, int64_t batch, double lr, uint64_t seed,
                           float* loss_hist);
/* One Adam step on a caller-given gradient (host [ADOT_MLP_PARAMS], packed as
 * adot_mlp_set_params), through the update kernel adot_mlp_train runs after
 * its backward pass: moments m, v updated with beta1 0.9, beta2 0.999, the
 * bias corrections of step t = (steps taken so far) + 1, eps 1e-8, step size
 * lr (0.05 + 0.95 (1 + cos(pi min(1, (t - 1) / total_steps))) / 2) (constant lr
 * when total_steps = 0), then the float32 master parameters and their bf16
 * copies; the step counter advances by one. Waits for the stream.
 * ADOT_E_INVALID_ARG for a NULL gradient, lr <= 0 or total_steps < 0. */
adot_status adot_mlp_apply_gradient(adot_mlp* mlp, const float* grad, double lr,
                                    int64_t total_steps);

/* Makes every later step of a float32 Grass context take |A|_Psi from the
 * network (A dW stays analytic), except on edges whose local Froude number
 * max(|Fr_L|, |Fr_R|, |Fr_mid|) lies in [fr_lo, fr_hi], whose two sides lie on
 * opposite sides of Fr = 1, or whose inputs leave the training box: those use
 * the analytic eigenstructure. mlp = NULL detaches. The network must outlive
 * its use by the context. ADOT_E_UNSUPPORTED for other contexts. */
adot_status adot_set_surrogate(adot_ctx* ctx, adot_mlp* mlp, double fr_lo, double fr_hi);
/* Edges evaluated and edges that fell back since the surrogate was attached. */
adot_status adot_surrogate_stats(adot_ctx* ctx, int64_t* edges_out, int64_t* fallback_out);
/* Evaluates the attached network on every edge 0..n of the current state
 * without stepping (the first half of a surrogate step). absA (may be NULL:
 * evaluate only) receives float32 [9][n+1]: row r holds entry r of the
 * row-major |A|_Psi, de-standardised; row 0 is NaN on the edges that take the
 * analytic eigenstructure instead, and *fallback_out (may be NULL) counts
 * them. Host or device pointer per on_device. Waits for the stream. Does not
 * change adot_surrogate_stats. ADOT_E_INVALID_ARG without a surrogate or a state. */
adot_status adot_surrogate_eval(adot_ctx* ctx, float* absA, int on_device, int64_t* fallback_out);
/* n edge samples of the current state (edge indices drawn with splitmix64 from
 * seed and the sample number): X [n][7] raw inputs and T [n][9] labels
 * |A|_Psi computed in float64, stored as float32 (host or device). Grass law. */
adot_status adot_harvest(adot_ctx* ctx, int64_t n, uint64_t seed, float* X, float* T, int on_device);

/* Largest number of cells adot_step_noalloc accepts. */
#define ADOT_NOALLOC_MAX_CELLS 65536

/* Allocation-free time stepping. The paper has no counterpart: this entry point
 * serves callers that cannot call cudaMalloc, such as a custom operation inside
 * another framework whose device memory must come from that framework's
 * allocator, or a real-time loop that reserves all memory before it starts.
 * It advances a caller-owned float64 state by n_steps steps of Eq. scheme and
 * allocates nothing, on the device or the host.
 *  - cfg: as for adot_create; precision must be ADOT_FP64 (else
 *    ADOT_E_UNSUPPORTED) and n_cells <= ADOT_NOALLOC_MAX_CELLS (else
 *    ADOT_E_INVALID_ARG). block_threads, reg_cap and steps_per_graph are
 *    ignored; cfg->device >= 0 is made current.
 *  - h, q, z: device arrays of n_cells float64, read and overwritten in place.
 *  - t_io: host pointer; the start time in, the time after the steps out.
 *  - cuda_stream: a cudaStream_t, or NULL for the legacy default stream. The call
 *    ends with a device-to-host read of the control block into host memory and
 *    cudaStreamSynchronize on that stream, and reports the first device-side
 *    error as adot_step does.
 * The second state buffer and the control block live in a file-scope device
 * array of ADOT_NOALLOC_MAX_CELLS cells (about 1.5 MB) that every GPU which
 * loads the library holds until the process exits. All calls share it: calls
 * that overlap on the GPU (on any stream or host thread) race, so callers must
 * serialise them; each call clears the control block before use.
 * Set-up: the first call on a device looks up the array's device address (once
 * per device, with that device current) and keeps it for the process. Under
 * CUDA's lazy module loading (the default) the driver places the array, and
 * each kernel this entry point runs, in the device's memory when they are first
 * used, not when the library is loaded. So the first call on a device is the
 * one that may allocate: make one call with the configuration you will use
 * (n_steps = 1 runs every kernel a longer call runs) before reserving the
 * device's memory, and before any stream capture. After that, calls with the
 * same configuration allocate nothing. A device reset (cudaDeviceReset) while
 * the library is loaded is not supported here: the address found at set-up
 * would no longer be valid. */
adot_status adot_step_noalloc(const adot_config* cfg, double* h, double* q, double* z,
                              int64_t n_steps, double* t_io, void* cuda_stream);

/* Throughput probe of one arithmetic pipe on a device (no counterpart in the
 * paper): the measured peaks that the step kernels' rooflines divide by. A
 * resident grid (8 blocks of 256 threads per SM) runs 8 independent chains
 * per thread; one warm-up launch, then one timed launch (CUDA events, tens of
 * milliseconds). kind: 0 = float32 FFMA (2 flops each), 1 = paired float32
 * FFMA2 (4 flops), 2 = MUFU reciprocal square root, 3 = MUFU sine, 5 = MUFU
 * float32 tanh (1 op each), 4 = float64 DFMA (2 flops), 6 = MUFU paired bfloat16
 * tanh (2 ops). *rate_out: flops (or ops) per second;
 * *seconds_out (may be NULL): the timed launch. device >= 0 is made current.
 * Allocates and frees a small result buffer and a stream.
 * ADOT_E_INVALID_ARG for another kind or a NULL rate_out. */
adot_status adot_measure_pipe(int kind, int device, double* rate_out, double* seconds_out);

/* Probe of the library's float32 device math for the tests (no counterpart in
 * the paper): y[i] = f(x[i]) for n values in device memory, on cuda_stream
 * (NULL = legacy stream), then waits for it. kind 0 = the step kernels'
 * arccos(x) / 3 (a degree-7 polynomial form of Abramowitz & Stegun 4.4.46,
 * evaluated in float32), kind 1 = CUDA's acosf(x) / 3. x in [-1, 1].
 * ADOT_E_INVALID_ARG for another kind, n < 0 or NULL arrays with n > 0. */
adot_status adot_math_probe(int32_t kind, const float* x, float* y, int64_t n, void* cuda_stream);

/* Name of a status code (static string). */
const char* adot_status_string(adot_status s);

/* Library version string (static). */
const char* adot_version(void);

#ifdef __cplusplus
}
#endif

#endif /* ADOT_H */
