/*
 * dds.h -- C ABI of libdds: trace-transfer diagonal sweeping domain decomposition for the
 * Helmholtz equation on one GB300 GPU (Leng & Ju, arXiv 2003.02585).
 *
 * Problem (Section 1, Eq. 1.1-1.2):  Delta u + kappa^2 u = f,  kappa(x) = omega / c(x),
 * truncated by the uniaxial PML of Eq. 2.1-2.3 (2D) / Eq. 4.1 (3D) and discretised with the
 * 5-point (2D) / 7-point (3D) second-order finite-difference stencil (Section 5).  The domain
 * is cut into an N1 x N2 [x N3] checkerboard (Section 2.3); every subdomain problem is extended
 * by its own PML (Lemma 2.3) with the wave number extended by Eq. 2.8, factored once, and the
 * 2^n diagonal sweeps of Algorithm 2.1 / Algorithm 4.1 are run with the trace routing of
 * Rules 2.4/2.5 (2D) and 4.1/4.2 (3D).
 *
 * Grid.  Cell-centred nodes x_p = (p + 1/2) h, p = 0..n_a-1 on the physical box [0, n_a h]
 * per axis, extended on every side by E = halo + pml_cells nodes (halo un-stretched lines, then
 * the PML), homogeneous Dirichlet just outside.  The "global extended grid" has
 * G_a = n_a + 2E nodes per axis.  Field arrays (f, u) are laid out [rhs][x3][x2][x1] over the
 * global extended grid, x1 fastest, as interleaved complex double (re, im) -- 16 bytes per node.
 *
 * PML profile (Eq. 2.1, profile left open by the paper): sigma(t) = S ((t - H h)/(P h))^power
 * for a distance t beyond the box edge larger than H h, alpha = 1 + i sigma.  The discrete
 * system is the J-scaled, complex-symmetric form A u = J f of Eq. 2.3 / 4.1, J = prod alpha.
 *
 * Pointers.  f, u, Au may be device pointers or host pointers (pageable or pinned); host
 * buffers are staged through device memory owned by the context.  The caller owns them; the
 * library never frees or retains a caller pointer after a call returns.
 *
 * Errors.  Every call returns a dds_status; nothing is thrown across the ABI.  On failure
 * dds_last_error(ctx) returns a message (valid until the next call on that context).  A context
 * may be used by one host thread at a time; a concurrent call returns DDS_EBUSY.
 */
#ifndef DDS_H
#define DDS_H

#ifdef __cplusplus
extern "C" {
#endif

typedef struct dds_ctx dds_ctx;

typedef enum {
  DDS_OK = 0,
  DDS_EINVAL = 1,    /* invalid argument (sizes, divisibility, null pointers)                */
  DDS_ENOMEM = 2,    /* device allocation failed or the memory budget would be exceeded       */
  DDS_ECUDA = 3,     /* a CUDA call failed (message holds the CUDA error string)              */
  DDS_ENOCONV = 4,   /* dds_solve reached maxit; u holds the best iterate                     */
  DDS_ETIMEOUT = 5,  /* a bounded device-side wait gave up                                    */
  DDS_EBUSY = 6      /* the context is in use by another thread                              */
} dds_status;

typedef enum {
  DDS_FP64 = 0,       /* every step in complex double                                         */
  DDS_MIXED = 1,      /* factors in FP64; sweeps (substitutions, trace transfer) in complex   */
                      /* single; FGMRES residual / orthogonalisation in FP64.  Substitutions  */
                      /* on the tensor cores as 3xTF32 split products (a b ~ a0 b0 + a0 b1 +  */
                      /* a1 b0, TF32 pieces, FP32 accumulation) where a line/plane block has  */
                      /* at most 128 nodes, FP32 CUDA cores otherwise                        */
  DDS_MIXED_BF16 = 2, /* as DDS_MIXED with BF16 pieces (16 K columns per MMA instead of 8;    */
                      /* about 4e-6 relative error per block product instead of 1e-6)         */
  DDS_MIXED_FP32 = 3  /* as DDS_MIXED with every substitution on the FP32 CUDA cores          */
} dds_precision;

typedef enum {
  DDS_PLAN_AUTO = 0,   /* trace-operator plan in 2D with lines of at most 128 nodes, direct   */
                       /* plan otherwise (3D, or wide 2D subdomains)                          */
  DDS_PLAN_DIRECT = 1, /* one batched local solve per (subdomain, RHS) per sweep step         */
  DDS_PLAN_TRACE = 2   /* local solves of the own sources and of the summed traces, sweep     */
                       /* steps through the precomputed trace-to-trace map (needs 16 T bytes  */
                       /* <= 200 KB, T = trace_len)                                           */
} dds_plan;

typedef struct {
  int dim;              /* 2 or 3                                                              */
  int n[3];             /* interior nodes per axis (n[2] ignored in 2D)                        */
  double h;             /* mesh width                                                          */
  double omega;         /* angular frequency; kappa = omega / c                                */
  const double *c;      /* wave speed at the n[0]*n[1]*(n[2]) interior nodes, x1 fastest;      */
                        /* HOST pointer, copied during dds_setup                               */
  int parts[3];         /* N1, N2 (, N3); n[a] % parts[a] == 0                                 */
  int pml_cells;        /* P >= 1                                                              */
  double pml_strength;  /* S (30 in the experiments of this library)                           */
  int pml_power;        /* profile exponent, 2 = quadratic                                     */
  int halo;             /* H >= 0 un-stretched lines between a box edge and its PML            */
  int precision;        /* dds_precision                                                       */
  int plan;             /* dds_plan                                                            */
} dds_problem;

typedef struct {
  int G[3];               /* global extended grid per axis                                    */
  int M[3];               /* extended subdomain grid per axis                                 */
  int n_sub;              /* number of subdomains                                             */
  int n_factors;          /* distinct extended-subdomain operators after deduplication        */
  int trace_len;          /* T: complex entries of all 2n two-line traces of one subdomain    */
  int plan;               /* plan in use                                                      */
  long long factor_bytes; /* device bytes held by factors (+ trace maps)                      */
  double setup_seconds;   /* wall time of dds_setup                                           */
  long long device_bytes; /* device memory the context holds now (dds_set_memory_budget)       */
  int trace_kernel;       /* trace solves: 0 = tensor cores (k_trace_tc), 1 / 2 = CUDA cores   */
                          /* with that many CTAs per SM (k_trace_sweeps), -1 = direct plan     */
  int subst_kernel;       /* substitutions: 0 = FP64 CUDA cores, 1 = FP32 CUDA cores,          */
                          /* 2 = tensor cores (lines <= 128 nodes), 3 = stage-parallel tensor  */
                          /* cores (wider blocks)                                              */
} dds_info_t;

/* dds_setup -- discretise, deduplicate and factor every extended subdomain (Section 2.3,
 * Eq. 2.8; block-tridiagonal LU over x_last lines/planes with partial pivoting inside each
 * Schur block, FP64 on the GPU) and allocate the sweep state.  *out receives a new context on
 * success and is left untouched on failure. */
dds_status dds_setup(const dds_problem *prob, dds_ctx **out);

/* dds_sweep, dds_solve and dds_apply take 1 <= nrhs <= 65535 right-hand sides per call
 * (DDS_EINVAL otherwise).
 *
 * dds_sweep -- the DDM as a direct solver: `rounds` rounds of the 2^n diagonal sweeps of
 * Algorithm 2.1 / 4.1 on the sources f (nrhs fields on the global extended grid), writing
 * u_DDM (Algorithm 2.1, last line) to u.  rounds >= 1 (Theorem 3.10 needs 2 in two-layer
 * media).
 *
 * Right-hand sides are independent: one whose source holds a NaN or infinite entry gets a NaN
 * field (dds_sweep, dds_sweep_strip) or a NaN field and relative residual (dds_solve, which then
 * returns DDS_ENOCONV); the other right-hand sides of the batch are computed as without it. */
dds_status dds_sweep(dds_ctx *ctx, const void *f, int nrhs, void *u, int rounds);

/* dds_sweep_strip -- the one-dimensional sweeping DDM of Section 3.2 on a strip partition
 * (exactly one axis a with N_a > 1, e.g. 1 x N2): nsweeps sweeps along axis a, forward (+)
 * first, then alternating, with the trace routing of Rules 2.4/2.5 (4.1/4.2) over that list and
 * u_DDM = sum of the sweeps' local solutions on owned nodes.  nsweeps = 2 is the forward and
 * backward sweep (the same field as dds_sweep with one round on the strip, whose other two
 * sweeps are empty); nsweeps = 3 adds the extra forward sweep of Theorem 3.6, which makes the
 * result exact (up to PML reflection) in two-layer media with an interface across the strip.
 * 1 <= nsweeps <= 64; DDS_EINVAL on a partition cut along more than one axis. */
dds_status dds_sweep_strip(dds_ctx *ctx, const void *f, int nrhs, void *u, int nsweeps);

/* dds_solve -- solve the discrete PML problem for nrhs sources with right-preconditioned
 * flexible GMRES, one DDM application (`rounds` rounds) per iteration as the preconditioner
 * (Section 5.2), FP64 residuals and orthogonalisation.  Stops when every RHS has relative
 * residual ||J f - A u|| / ||J f|| < tol or after maxit iterations (then DDS_ENOCONV).
 * iters (may be NULL) receives the iteration count; relres (may be NULL, else nrhs doubles,
 * host memory) the final true relative residual of each RHS. */
dds_status dds_solve(dds_ctx *ctx, const void *f, int nrhs, void *u, double tol, int maxit,
                     int rounds, int *iters, double *relres);

/* dds_apply -- Au = J^{-1} A u: the PML operator L of Eq. 2.3 / 4.1 applied to nrhs fields
 * (so that dds_apply(dds_solve(f)) ~= f). */
dds_status dds_apply(dds_ctx *ctx, const void *u, int nrhs, void *Au);

/* dds_local_solve -- one block-tridiagonal subdomain solve A_R x = b (the local problem
 * P_{Omega_ij, kappa_ij} of Algorithm 2.1), for nrhs right-hand sides b laid out
 * [rhs][x3][x2][x1] over the extended subdomain grid (M per axis), interleaved complex double.
 * sub is the subdomain's linear index (x1 fastest).  Runs in the context's precision.
 * DDS_ETIMEOUT if a bounded device-side wait in the substitutions gave up. */
dds_status dds_local_solve(dds_ctx *ctx, int sub, const void *b, int nrhs, void *x);

/* dds_local_solve_noalloc -- dds_local_solve for callers that must not have this library
 * allocate device memory.  The paper has no counterpart; this is a deployment variant.
 * Who needs it: a host program whose device memory is fully reserved by another allocator (a
 * framework's caching allocator, a fixed serving budget), where a cudaMalloc inside the call
 * would fail or evict that allocator's cache, or a latency-critical caller that cannot accept
 * the device-wide synchronisation cudaMalloc / cudaFree may cause.
 * Contract: b and x are DEVICE pointers on the context's device (host pointers are rejected
 * with DDS_EINVAL, since staging them would need a buffer).  All scratch -- the working copy of
 * the right-hand sides and the launch descriptors -- lives in one fixed 8 MiB array compiled
 * into the library (every GPU that loads libdds holds it until the process exits): at most 256
 * right-hand sides and nrhs * M^n * (16 bytes in DDS_FP64, 8 in DDS_MIXED) <= 8 MiB - 16 KiB,
 * larger requests return DDS_EINVAL with the sizes in dds_last_error.  The call makes no
 * cudaMalloc / cudaFree.  The first call on a device looks up the array's device address (once
 * per device, with that device current); make that first call before any stream capture.
 * Every call on a device shares the one array and leaves its contents behind: calls that
 * overlap on the GPU (other contexts or streams on the same device) race on it.  The call
 * waits for its stream before it returns; DDS_ETIMEOUT if a bounded device-side wait in the
 * substitutions gave up (x is then not valid). */
dds_status dds_local_solve_noalloc(dds_ctx *ctx, int sub, const void *b, int nrhs, void *x);

/* ---- continuous-batching server (serving several requests against one set-up context) ------
 * A server owns max_slots right-hand-side slots, each running its own right-preconditioned
 * FGMRES (the dds_solve algorithm).  dds_server_step admits queued right-hand sides into free
 * slots, applies ONE batched DDM application (`rounds` rounds) to the current Krylov vector of
 * every active slot, completes that iteration's FP64 Arnoldi step per slot, and retires slots
 * whose relative residual is below tol (or that reached maxit).  Requests submitted while others
 * are in flight therefore join at the next iteration.  Slot memory ((2 maxit + 5) fields per
 * slot, and the slot's columns of the batched DDM's work buffers) is allocated by
 * dds_server_create, which admits by device memory: it takes as many slots as fit in the room
 * the context's budget leaves (dds_set_memory_budget; without a budget, 90% of the device's
 * free memory), at most max_slots, and returns DDS_ENOMEM if not even one fits.  The slot
 * count is the admission limit (dds_server_slots).  Destroy a server before its context. */
typedef struct dds_server dds_server;

dds_status dds_server_create(dds_ctx *ctx, int max_slots, double tol, int maxit, int rounds,
                             dds_server **out);

/* slots of a server (its admission limit) */
int dds_server_slots(const dds_server *srv);

/* queue one source field f (global extended grid, complex double, host or device); tag is
 * returned with its solution.  The field is copied before the call returns: into device memory
 * while the context's budget (dds_set_memory_budget) has room for it beyond the eighth the
 * server keeps free for its steps, otherwise (or when the device has no room) into host memory,
 * from which admission copies it to its slot.  DDS_ENOMEM only if neither has room. */
dds_status dds_server_submit(dds_server *srv, const void *f, long long tag);

/* one batched iteration; *active = slots in flight after it, *queued = requests still waiting */
dds_status dds_server_step(dds_server *srv, int *active, int *queued);

/* pop one finished request: tag, solution u (host or device, one field), FGMRES iterations and
 * final true relative residual.  Returns DDS_EBUSY (and touches nothing) when none is ready. */
dds_status dds_server_poll(dds_server *srv, long long *tag, void *u, int *iters, double *relres);

/* free the server.  The server may outlive its context: dds_destroy releases the device memory
 * of every server made on the context and leaves them orphaned; every later call on an orphaned
 * server but this one returns DDS_EINVAL. */
void dds_server_destroy(dds_server *srv);

/* dds_set_stream -- run all later work of ctx on the given cudaStream_t (NULL = the context's
 * own stream).  Calls still return only after their work has completed. */
dds_status dds_set_stream(dds_ctx *ctx, void *cuda_stream);

/* dds_get_info -- sizes and counts of a set-up context. */
dds_status dds_get_info(const dds_ctx *ctx, dds_info_t *info);

/* dds_kernel_launches -- number of kernels this context has launched so far. */
long long dds_kernel_launches(const dds_ctx *ctx);

/* dds_autotune -- time the tunable launch shapes of one DDM application on this context's
 * geometry for nrhs right-hand sides and `rounds` rounds, and keep the fastest:
 *   the tensor-core substitution panel width (8, 16 or 32 columns) and panels per CTA or CTA
 *   pair (1, or 2 for widths up to 16: one panel's epilogue runs under the other's MMAs;
 *   mixed modes with tensor-core substitutions), and the trace-solve kernel of the trace plan:
 *   the CUDA-core cooperative launch with 1 or 2 CTAs per SM, or (0) the tensor-core launch
 *   (split products of the context's piece type; mixed modes with tensor-core pieces).
 * Each candidate is captured once and then timed over three DDM applications with CUDA events
 * on the context's stream, with synthetic nonzero right-hand sides in scratch the call allocates
 * and frees.  table (row-major [n][4]: panel width (0 = automatic), panels per CTA, trace
 * kernel (CTAs per SM of the CUDA-core launch, 0 = tensor cores), ms per DDM application)
 * receives at most max_entries rows; *n_entries is the number of candidates timed; best[0],
 * best[1], best[2] (three ints) the chosen panel width, trace kernel and panels per CTA.  Cached plans and graphs are dropped.
 * Not part of the paper: it picks block and panel tile shapes by measurement. */
dds_status dds_autotune(dds_ctx *ctx, int nrhs, int rounds, int max_entries, int *n_entries,
                        double *table, int *best);

/* dds_set_launch_shape -- set the tunable launch shapes directly (the values dds_autotune
 * chooses, so that a measured choice can be pinned): panel_width 8, 16 or 32 (0 = automatic)
 * and panels_per_cta 1 or 2 of the tensor-core substitutions, trace_kernel 0 (tensor cores) or
 * 1 / 2 (CUDA cores, CTAs per SM).  DDS_EINVAL for a shape this context cannot run.  Drops cached
 * plans and graphs. */
dds_status dds_set_launch_shape(dds_ctx *ctx, int panel_width, int panels_per_cta,
                                int trace_kernel);

/* dds_tensor_rate -- measured dense tensor-core rate of the current device for a split-product
 * piece type: kind 0 = TF32 (tcgen05 kind::tf32), 1 = BF16 (kind::f16), in TFLOP/s of the
 * pieces (a 3x split product delivers a third of it in useful flops).  Every SM issues
 * back-to-back M = 128, N = 256 MMAs from shared memory into tensor memory for about a
 * millisecond, as the substitution and trace kernels do.  Needs no context; runs on its own
 * stream and synchronises it.  DDS_EINVAL for another kind, DDS_ETIMEOUT if the completion wait
 * gave up, DDS_ECUDA on a CUDA error. */
dds_status dds_tensor_rate(int kind, double *tflops);

/* dds_work_per_ddm -- algorithmic floating-point work of one DDM application (Algorithm 2.1 /
 * 4.1, `rounds` rounds of 2^n sweeps) for nrhs right-hand sides, computed on the host:
 *   *subst_flops  block forward + back substitutions, 16 Ml Mb^2 real flops per local solve
 *                 (2 Ml Mb^2 complex multiply-adds), times the local solves of the plan;
 *   *trace_flops  trace-map applications of the trace plan: 8 x (map rows of routed sides that
 *                 have a neighbour) x (inputs of receiving sides that have one) per (sweep,
 *                 subdomain, RHS); 0 for the direct plan.
 * Used to turn kernel times into achieved rates.  DDS_EINVAL on bad arguments. */
dds_status dds_work_per_ddm(dds_ctx *ctx, int nrhs, int rounds, double *subst_flops,
                            double *trace_flops);

/* dds_set_memory_budget -- cap the device memory this context may hold: its factors and trace
 * maps, work buffers, launch tables, staging buffers and the slots of its servers.  A call whose
 * allocations would take the total above `bytes` returns DDS_ENOMEM (with the sizes in
 * dds_last_error) and leaves the context usable for smaller calls; buffers already held stay.
 * 0 removes the cap.  *in_use (may be NULL) receives the bytes held now.  A real cudaMalloc
 * failure returns DDS_ENOMEM the same way.  Not part of the paper: admission control for a
 * device shared by several contexts or servers. */
dds_status dds_set_memory_budget(dds_ctx *ctx, long long bytes, long long *in_use);

/* dds_set_wait_limit -- polls a level-completion wait of the cooperative trace launches makes
 * before it gives up (the launch then ends with wrong results and the call returns
 * DDS_ETIMEOUT); 0 restores the default (2^20 polls, about 0.1 s).  A diagnostic control: a
 * small limit makes those waits run out on purpose (no GPU fault, the context stays usable),
 * which is how the timeout path is tested.  Drops cached CUDA graphs. */
dds_status dds_set_wait_limit(dds_ctx *ctx, long long polls);

/* dds_set_zero_skip -- zero-work skipping (Algorithm 2.1: a subdomain whose assembled right-hand
 * side f_ij is zero is not solved, u_ij = 0).  On (enable = 1, the default), after each batched
 * assembly the (subdomain, RHS) local problems whose right-hand side is exactly zero are dropped
 * from the substitution launch on the device (their solution is the zero already in place); the
 * result is the same as with skipping off (bit-identical in DDS_FP64).  Off (0) solves every
 * local problem, e.g. to compare.  Drops cached CUDA graphs when it changes the setting. */
dds_status dds_set_zero_skip(dds_ctx *ctx, int enable);

/* dds_local_solve_counts -- (subdomain, RHS) local problems whose substitutions ran (*solved)
 * and that were assembled (*assembled) in the DDM applications of dds_sweep, dds_sweep_strip,
 * dds_solve and the server since the context was set up or last reset; with zero-work skipping
 * off both count only the compacted launches (0).  reset != 0 zeroes the counts after reading.
 * Synchronises the context's stream. */
dds_status dds_local_solve_counts(dds_ctx *ctx, long long *solved, long long *assembled,
                                  int reset);

/* Kernel families timed by the profiler (dds_profile_read). */
typedef enum {
  DDS_K_ASSEMBLE = 0,   /* own-source + trace-potential right-hand sides                    */
  DDS_K_SUBST = 1,      /* block-tridiagonal forward + back substitution                    */
  DDS_K_EXTRACT = 2,    /* own-node accumulation, trace extraction and routing              */
  DDS_K_TRACE_STEP = 3, /* trace-operator sweep step (trace plan)                            */
  DDS_K_KRYLOV = 4,     /* FP64 operator apply, reductions and vector updates               */
  DDS_K_OTHER = 5,      /* set-up, conversions                                              */
  DDS_K_COUNT = 6
} dds_kernel_kind;

/* dds_profile -- enable (1) / disable (0) per-launch CUDA-event timing on the context's
 * stream.  Enabling clears the accumulated statistics. */
dds_status dds_profile(dds_ctx *ctx, int enable);

/* dds_profile_read -- launches and summed device milliseconds of one kernel family since
 * profiling was enabled (synchronises the context's stream). */
dds_status dds_profile_read(dds_ctx *ctx, int kind, long long *launches, double *ms);

/* dds_last_error -- message of the last failed call on ctx (empty string if none). */
const char *dds_last_error(const dds_ctx *ctx);

/* dds_destroy -- free every device and host resource of ctx (NULL is ignored), including the
 * device memory of the servers made on it, which stay allocated as orphans until
 * dds_server_destroy. */
void dds_destroy(dds_ctx *ctx);

#ifdef __cplusplus
}
#endif
#endif /* DDS_H */
