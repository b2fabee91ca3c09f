/*
 * rt.h - C interface of the GB300 photon-transport library (librt_gb300.so).
 *
 * The library advances the two-moment radiation equations (photon energy density E
 * and flux F per photon group, M1 closure, reduced speed of light c) on static
 * finite-volume particles, as in GEAR-RT (Ivkovic 2023, arXiv 2302.12727, Part III,
 * chapter "One RT Time Step"):
 *
 *   injection:   E_g += xi_sg L_s dt / V_g        (Sec. "First step: Injection",
 *                                                  Eq. isotropy-correction-with-zero)
 *   transport:   U_k(t+dt) = U_k - dt/V_k sum_l F_kl . A_kl
 *                                                 (Eq. transport-update-explicit, Eq. rt-meshless)
 *                with A_kl the Hopkins effective surfaces (Eq. HopkinsAij), gradients from
 *                the least-squares estimate (Eqs. gradient, psitilde, matrix_B, matrix_E),
 *                minmod-limited states at x_kl (Eq. rt-riemann-problem, Eq. rt-minmod)
 *                and the GLF flux (Eq. riemann-GLF) of the M1 closure (Eq. eddington-group);
 *   sink:        U <- U max(0, 1 - c alpha dt)    (Sec. "Third step: Thermochemistry",
 *                                                  forward-Euler photon removal, grey alpha)
 *
 * Conventions shared by every entry point:
 *  - Array arguments named *_dev are DEVICE pointers owned by the caller, in the caller's
 *    particle order.  Multi-component arrays are component-major (structure of arrays):
 *      x     [3][N]        positions (double)
 *      U     [G][4][N]     (E, Fx, Fy, Fz) per group; element type double for RT_FP64,
 *                          float for RT_FP32_MIXED
 *      gradU [G][4][3][N]  d/dx, d/dy, d/dz of each component; element type as U
 *      Lsrc  [S][G]        source luminosities (double)
 *      alpha [N]           grey absorption coefficient (double), or NULL for none
 *  - The library owns its workspaces, its cell-sorted copies and the permutation.  Memory is
 *    allocated only in rt_create, rt_neighbours and on the first call of rt_adjoint with a
 *    larger checkpoint count; rt_transport_step and rt_subcycle allocate nothing.
 *  - All work is asynchronous on the stream given to rt_create, except where a function
 *    says it synchronises.  Nothing aborts or prints: every call returns an rt_status and
 *    rt_last_error() gives a message for the last failure.
 *  - rt_neighbours must be called before any transport call (else RT_ERR_STATE); its
 *    geometry is kept until the next rt_neighbours.
 */
#ifndef RT_GB300_RT_H
#define RT_GB300_RT_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct rt_ctx rt_ctx;

/* Riemann solvers of the pair flux (rt_config.riemann_solver). */
enum { RT_RIEMANN_GLF = 0, RT_RIEMANN_HLL = 1 };

/* Size of the HLL wave-speed table: RT_WAVE_NF values of f = i / (RT_WAVE_NF - 1) by
 * RT_WAVE_NTH values of theta = j pi / (RT_WAVE_NTH - 1). */
#define RT_WAVE_NF 101
#define RT_WAVE_NTH 101

typedef enum {
    RT_OK = 0,
    RT_ERR_INVALID = 1,   /* bad argument or configuration */
    RT_ERR_CUDA = 2,      /* a CUDA call failed; the message names it */
    RT_ERR_OOM = 3,       /* device allocation failed */
    RT_ERR_NOCONV = 4,    /* smoothing-length iteration did not converge */
    RT_ERR_GEOMETRY = 5,  /* singular E_i (fewer than 3 non-coplanar neighbours) or
                             a support radius of half the periodic box or more */
    RT_ERR_TIMEOUT = 6,   /* a bounded device wait ran out */
    RT_ERR_STATE = 7      /* call out of order (e.g. transport before rt_neighbours) */
} rt_status;

enum { RT_FP64 = 0, RT_FP32_MIXED = 1 };

typedef struct {
    int32_t n_groups;        /* G >= 1 photon groups; transport treats them independently */
    double c_red;            /* reduced speed of light, used in the closure, the GLF
                                dissipation and the sink (Sec. reduced speed of light) */
    double eta_res;          /* resolution parameter of the gas h, 1.2348 gives ~48 neighbours
                                (Eq. number-of-neighbors) */
    double eta_res_star;     /* the same for the sources' injection radius */
    double box[3];           /* box side lengths; positions must lie in [0, box) */
    int32_t periodic;        /* 1: periodic box, minimal-image separations */
    int32_t precision;       /* RT_FP64: everything in double.  RT_FP32_MIXED: fluxes and
                                gradients in float; h, E_i, B_i = E_i^-1 and the energy sum in
                                double */
    int32_t clamp_negative;  /* 1: set E < 0 to 0 after each step (counted); breaks exact
                                conservation, so 0 for conservation checks */
    int32_t limiter_variant; /* 0: s = minmod(grad Q_k . d, grad Q_l . d) on both states (the only
                                value accepted) */
    double h_tol;            /* relative tolerance of the float phase of the smoothing-length
                                iteration (<= 1e-6); both precisions then refine h in double to
                                machine precision, so they share one neighbour set */
    int32_t h_max_iter;      /* iteration cap of that solve; exceeding it gives RT_ERR_NOCONV */
    uint64_t device_wait_budget_cycles;  /* bound, in SM clock cycles, of every device-side wait
                                            (the copy waits of flux_variant 2, rt_tuning); 0 means
                                            4e9 (about two seconds).  A wait that runs out skips
                                            its pairs and sets a flag that rt_energy reports as
                                            RT_ERR_TIMEOUT (and rt_diag.wait_timeouts) until the
                                            next rt_neighbours */
    int32_t riemann_solver;  /* RT_RIEMANN_GLF (Eq. riemann-GLF) or RT_RIEMANN_HLL (Eq. riemann-HLL:
                                wave speeds from the library's M1 eigenvalue table, see
                                rt_wave_table); rt_adjoint supports GLF only */
} rt_config;

typedef struct {
    int64_t n_pairs;          /* unordered interacting pairs P (r < max(H_i, H_j)) */
    int64_t n_directed;       /* entries of the symmetric neighbour lists, 2P */
    int64_t n_injection;      /* (source, gas) injection entries */
    int64_t n_ill_conditioned;/* particles with cond_2(E_i) > 1e10 */
    double cond_max;          /* largest cond_2(E_i) */
    double h_min, h_max;      /* smoothing lengths */
    double dx_min;            /* min_i (V_i / (4 pi / 3))^(1/3), the cell size of Eq. rt-cfl */
    int64_t clamp_events;     /* cumulative count of E < 0 fix-ups */
    int32_t grid[3];          /* cell-list dimensions used by rt_neighbours */
    int32_t threads_per_particle;  /* threads per particle of the float gradient kernel (G,
                                      at most 4, in gradient_variants 1 and 2; else 1) */
    int64_t kernel_launches;  /* cumulative launches of the library's own kernels (graph
                                 replays count every kernel node; library sorts and scans
                                 that the build calls are not counted) */
    int32_t pair_build;       /* pair-list build of the last rt_neighbours: 0 = every particle
                                 searched to max(H_i, H_max); 1 = own supports, then sorted and
                                 de-duplicated with their transposes (chosen when the h range is
                                 wide); both give the same lists */
    int32_t wait_timeouts;    /* 1 if a device-side wait ran out since the last rt_neighbours */
    int64_t h_refined;        /* particles whose h the last rt_neighbours refined in double: all of
                                 them on the FP64 path; on the float path those with a neighbour
                                 candidate within 1e-4 of their support radius at the float root */
} rt_diag;

/* Launch variants of the float (RT_FP32_MIXED) pair kernels.  The paper has no counterpart:
 * they choose how the GPU threads map onto the pair loops of Eq. gradient and
 * Eq. transport-update-explicit, never what is computed.  Every variant gives bitwise the
 * same fluxes and the same order of accumulation; the double path ignores them (but not
 * cell_eighths).
 *   flux_variant      0: one thread per pair slot loading both particles' records directly;
 *                     1: the same, with the neighbour records of each warp staged through
 *                        shared memory by cooperative asynchronous copies;
 *                     2: the same, with the neighbour rows of each warp fetched into shared
 *                        memory by tensor-memory-accelerator row gathers (default; falls back
 *                        to 0 where the CUDA driver offers no tensor-map encoder).
 *   gather_variant    0: one thread per particle;
 *                     1: one thread per (particle, group) (default).
 *   gradient_variant  0: one thread per particle;
 *                     1: one thread per (particle, group);
 *                     2: one thread per (particle, group), the lanes of a particle
 *                        computing the neighbour separations and kernel weights once between
 *                        them and exchanging them by warp shuffles (default; as 1 for one
 *                        group).
 * Changing the variants drops the context's captured sub-cycle graphs. */
typedef struct {
    int32_t flux_variant;
    int32_t gather_variant;
    int32_t gradient_variant;
    /* Launch shapes and the cell list (also bitwise neutral, except cell_eighths):
     *   cell_eighths    edge of the neighbour search's cells, in eighths of the support
     *                   radius at the mean density, kappa eta (box volume / N)^(1/3): 2 to 16
     *                   (default 4).  It applies from the next rt_neighbours and changes the
     *                   cell-sorted order, hence the order of the neighbour sums: the results
     *                   then differ by rounding, the pair lists not at all.
     *   gradient_block  threads per block of the float gradient kernels: 32, 64, 128 or 256;
     *                   0 = the variant's default (64 for variant 2, 256 for variant 1).
     *   gather_block    threads per block of gather_variant 1: a multiple of 32 from 64 to 512;
     *                   0 = 256.
     *   pair_warps      warps per block of flux_variant 2: 1, 2 or 4; 0 = 1. */
    int32_t cell_eighths;
    int32_t gradient_block;
    int32_t gather_block;
    int32_t pair_warps;
} rt_tuning;

/* Kernel kinds reported by rt_kernel_times. */
enum { RT_KERNEL_INJECT = 0, RT_KERNEL_GRADIENT = 1, RT_KERNEL_FLUX = 2, RT_KERNEL_FLUX_GATHER = 3,
       RT_KERNEL_KINDS = 4 };

/* Create a context for n particles and n_src sources.  cuda_stream is a cudaStream_t
 * (NULL = legacy default stream).  Allocates the per-particle workspaces.  On failure
 * *out is still set (so rt_last_error can be read) unless out is NULL; destroy it. */
rt_status rt_create(const rt_config* cfg, int64_t n, int64_t n_src, void* cuda_stream, rt_ctx** out);

/* Change the stream used by later calls. */
rt_status rt_set_stream(rt_ctx* ctx, void* cuda_stream);

/* Neighbour search and geometry, once per particle configuration (Part II, "The Neighbor
 * Search"; Eqs. omega, particle-volume, matrix_E, matrix_B; sources: Sec. "Weights For
 * Distribution Of Energy Density of a Star onto Particles"):
 * cell-list build, smoothing lengths h_i = eta omega_i^(-1/3), the symmetric pair lists
 * { j : r_ij < max(H_i, H_j) }, H = 1.825742 h, E_i and B_i = E_i^-1 in double, source
 * radii and injection weights.
 *   x_dev    [3][N] positions in [0, box)
 *   m_dev    [N] masses (kept for the caller's density; may be NULL)
 *   xsrc_dev [3][S] source positions (may be NULL when S = 0)
 *   h_out    [N] device, receives h_i in caller order (may be NULL)
 * Synchronises the stream (it sizes the pair lists).  Errors: RT_ERR_INVALID (NaN/Inf or
 * out-of-box positions), RT_ERR_NOCONV, RT_ERR_GEOMETRY, RT_ERR_OOM. */
rt_status rt_neighbours(rt_ctx* ctx, const double* x_dev, const double* m_dev, const double* xsrc_dev,
                        double* h_out_dev);

/* The neighbour search of rt_neighbours with the smoothing lengths given instead of solved:
 * h_dev [N] (caller order) for the gas and hs_dev [S] for the sources (NULL when S = 0),
 * device doubles, read during the call.  omega_i = sum_j W(r_ij, h_i) is evaluated at the
 * given h_i (in the working precision's arithmetic of the solve's last iteration), and the
 * pair lists, E_i, B_i and the injection weights follow as in rt_neighbours.  This is the
 * build of a rank in a spatial domain decomposition (Part II, "Distributed Memory
 * Parallelism: Domain Decomposition and MPI"): the owner of a particle solves its h with a
 * complete neighbourhood and sends it to the ranks holding the particle as a ghost, so that
 * every rank decides the pairs of its particles with the same h.  RT_ERR_INVALID for NULL
 * arrays or an h that is not finite and positive (or, periodic box, reaches half the box
 * with its support); other errors as rt_neighbours. */
rt_status rt_neighbours_given_h(rt_ctx* ctx, const double* x_dev, const double* m_dev, const double* xsrc_dev,
                                const double* h_dev, const double* hs_dev);

/* As rt_neighbours_given_h, with each source's omega_s (omegas_dev [S]) and octant sums
 * w_a (octw_dev [S][8]) given too (Sec. "Weights For Distribution Of Energy Density", Eq.
 * isotropy-correction-with-zero), device doubles read during the call: the weights xi_sg
 * of the gas this context holds are then the ones the whole set gives, however much of the
 * source's support it holds.  A rank of a domain decomposition takes them from the source's
 * owner (the thesis's star send/recv), so that it needs no gas halo for the injection.  All
 * four arrays may be NULL only when S = 0; errors as rt_neighbours_given_h. */
rt_status rt_neighbours_given_fields(rt_ctx* ctx, const double* x_dev, const double* m_dev, const double* xsrc_dev,
                                     const double* h_dev, const double* hs_dev, const double* omegas_dev,
                                     const double* octw_dev);

/* Smoothing lengths h_s of the sources from the last rt_neighbours (hs_dev [S], device
 * doubles, source order as given; written asynchronously on the context's stream). */
rt_status rt_source_fields(rt_ctx* ctx, double* hs_dev);

/* Each source's omega_s (omegas_dev [S]) and octant sums w_a (octw_dev [S][8]) from the
 * last rt_neighbours, device doubles, written asynchronously; nothing when S = 0. */
rt_status rt_source_norms(rt_ctx* ctx, double* omegas_dev, double* octw_dev);

/* Particles owned by this context: caller indices [0, n_owned); the rest are ghost copies of
 * particles another rank owns (a domain decomposition places them last).  rt_energy then
 * sums the owned particles only; the transport still updates every particle (a ghost's new
 * state is discarded by its next refresh from the owner).  n_owned = n (the default) owns
 * all.  RT_ERR_INVALID outside [0, n]. */
rt_status rt_set_owned(rt_ctx* ctx, int64_t n_owned);

/* Least-squares gradients of every component of U (Eq. gradient):
 * grad Q_i = sum_j (Q_j - Q_i) psitilde_j(x_i).  U_dev [G][4][N], gradU_dev [G][4][3][N]. */
rt_status rt_gradients(rt_ctx* ctx, const void* U_dev, void* gradU_dev);

/* One time step dt: injection, transport, sink (and fix-up if enabled), in place on U_dev.
 * Lsrc_dev may be NULL when S = 0; alpha_dev may be NULL (no sink).  Plain kernel launches. */
rt_status rt_transport_step(rt_ctx* ctx, double dt, void* U_dev, const double* Lsrc_dev, const double* alpha_dev);

/* The injection stage of one step alone (Sec. "Weights For Distribution Of Energy
 * Density"): E_g += sum_s xi_sg Lsrc_s,g dt / V_g over the injection targets, in place on
 * U_dev ([G][4][N], caller order, element type per precision; device).  Lsrc_dev [S][G]
 * (double, device) may be NULL, and with it, with S = 0 or with no targets, the call
 * changes nothing.  rt_inject followed by rt_transport_step with Lsrc_dev = NULL gives
 * bitwise the result of rt_transport_step with Lsrc_dev (the same injection kernel on the
 * same values).  RT_ERR_INVALID for a NULL U_dev or a dt that is negative or not finite. */
rt_status rt_inject(rt_ctx* ctx, double dt, void* U_dev, const double* Lsrc_dev);

/* The transport and sink of one step (Eqs. transport-update-explicit, riemann-GLF or
 * riemann-HLL, and the sink) with the gradients given instead of computed: gradU_dev
 * [G][4][3][N] in caller order, element type per precision (as rt_gradients writes them);
 * no injection.  With gradU_dev from rt_gradients on the same U_dev it gives bitwise the
 * result of rt_transport_step without sources.  A domain decomposition that exchanges
 * gradients (the thesis's RT gradient send/recv) supplies its ghosts' gradients from their
 * owners this way.  Plain launches; RT_ERR_INVALID for NULL arrays or a bad dt. */
rt_status rt_transport_step_given_gradients(rt_ctx* ctx, double dt, void* U_dev, const void* gradU_dev,
                                            const double* alpha_dev);

/* Per-particle fields of caller particles [first, first + count) given instead of the
 * context's own (Eqs. omega, particle-volume, matrix_B): omega_dev [count] and B_dev
 * [count][3][3] (double, device, caller order); V = 1 / omega follows, and the pair
 * kernels' records are derived from them as the neighbour search derives its own.  Valid
 * until the next rt_neighbours.  A rank of a domain decomposition gives its ghosts the
 * fields their owners computed with complete neighbourhoods.  RT_ERR_INVALID for a range
 * outside [0, N) or NULL arrays with count > 0. */
rt_status rt_set_fields(rt_ctx* ctx, int64_t first, int64_t count, const double* omega_dev, const double* B_dev);

/* n_sub steps of size dt without any neighbour search in between (Sec. "Dynamic
 * Sub-Cycling"), replayed from one CUDA graph that the library captures once per
 * (n_sub, source/sink presence) and reuses; dt, Lsrc and alpha live in device buffers,
 * so they may change between calls without a new capture. */
rt_status rt_subcycle(rt_ctx* ctx, int32_t n_sub, double dt, void* U_dev, const double* Lsrc_dev,
                      const double* alpha_dev);

/* Reverse-mode derivative of rt_subcycle (no counterpart in the thesis): given
 * dL/dU(final) it returns dL/dU0 [G][4][N] and dL/dLsrc [S][G] (double, may be NULL).
 * The forward pass keeps a checkpoint every ckpt_every steps and recomputes each segment
 * in reverse.  U0_dev is not modified.  The fix-up (clamp_negative) is treated as inactive. */
rt_status rt_adjoint(rt_ctx* ctx, int32_t n_sub, double dt, int32_t ckpt_every, const void* U0_dev,
                     const double* Lsrc_dev, const double* alpha_dev, const void* dLdU_final_dev,
                     void* dLdU0_dev, double* dLdLsrc_dev);

/* Individual time bins (Part II Sec. "Individual Timstepping", Eq. transport-update-explicit
 * with min(dt_k, dt_l); Part III Sec. "Dynamic Sub-Cycling").  Particle i advances in steps
 * dt_i = 2^b_i dt_min; a hydro step is 2^B min-steps, B = max_i b_i.  At min-step s particle i
 * starts a step when s mod 2^b_i = 0: it takes its injection over dt_i and a new gradient
 * (the others keep theirs); every pair with a starting member exchanges the time-integrated
 * flux min(dt_k, dt_l) F_kl . A_kl into both particles' accumulators; at the end of its
 * step particle i applies U_i - acc_i / V_i, then its sink over dt_i (grey or per group)
 * and the fix-up.  The exchange is antisymmetric, so the total energy is conserved.
 *
 * rt_set_time_bins: bins from bins_dev (N int32, caller order, clipped to [0, max_bin]) or,
 *   with bins_dev == NULL, from each particle's CFL step (Eq. rt-cfl): the largest
 *   b <= max_bin with 2^b dt_min <= cfl dx_i / c, dx_i = (V_i / (4 pi / 3))^(1/3); then, if
 *   `limit`, the limiter lowers them until neighbours differ by at most 2 bins (a factor 4
 *   in time step).  Call after rt_neighbours (which discards the bins).  Synchronises.
 * rt_get_time_bins: the bins in use (bins_dev: N int32, caller order, may be NULL) and B.
 * rt_step_bins: one hydro step (2^B min-steps, plain launches) on U_dev (4G x N, caller
 *   order, in/out) with luminosities Lsrc_dev (S x G or NULL) and grey absorption alpha_dev
 *   (N or NULL; the per-group absorbers of rt_set_absorbers apply when NULL).  Every bin 0
 *   gives one rt_transport_step of dt_min.
 * RT_ERR_STATE before rt_neighbours or without bins; RT_ERR_INVALID for a non-positive
 * dt_min, max_bin outside [0, RT_MAX_TIME_BIN] or a missing cfl. */
#define RT_MAX_TIME_BIN 20
rt_status rt_set_time_bins(rt_ctx* ctx, const int32_t* bins_dev, double dt_min, double cfl, int32_t max_bin,
                           int32_t limit);
rt_status rt_get_time_bins(rt_ctx* ctx, int32_t* bins_dev, int32_t* max_bin_host);
rt_status rt_step_bins(rt_ctx* ctx, void* U_dev, const double* Lsrc_dev, const double* alpha_dev);

/* Drift correction (Sec. "Dealing With Particle Drifts"): particles that the hydrodynamics
 * moves by dx_i = v_i dt_drift take the state extrapolated with their least-squares
 * gradient (Eq. gradient) at the old position, U_i <- U_i + grad U_i . dx_i, for every
 * component of every group.  U_dev (4G x N, caller order, element type per precision) is
 * read and overwritten; v_dev (3 x N doubles, caller order, component-major) is read only.
 * The gradients are those of the current (old) particle set, so call rt_drift before
 * rt_neighbours with the moved positions.  Like the thesis's scheme it does not conserve
 * the total energy exactly.  RT_ERR_STATE before rt_neighbours; RT_ERR_INVALID for NULL
 * arrays or a non-finite dt_drift. */
rt_status rt_drift(rt_ctx* ctx, void* U_dev, const double* v_dev, double dt_drift);

/* Total radiation energy per group, sum_i V_i E_i,g, summed in double in a fixed order over
 * the owned particles (all of them unless rt_set_owned says otherwise).
 * E_tot_host [G] is HOST memory; the call synchronises the stream. */
rt_status rt_energy(rt_ctx* ctx, const void* U_dev, double* E_tot_host);

/* Total radiation energy per group, sum_i V_i E_i,g, without allocating anything and
 * without a context.  The thesis has no counterpart: this entry point exists for callers
 * that must not allocate device memory themselves or through the library, such as a host
 * simulation code whose memory pool owns the whole GPU and forbids other allocations, or
 * a monitoring hook that has to leave device memory untouched.
 *   U_dev      [G][4][N] state in caller order (double for RT_FP64, float for RT_FP32_MIXED)
 *   V_dev      [N] particle volumes in caller order (double), e.g. from rt_particle_fields
 *   n          number of particles (>= 1)
 *   n_groups   G, at most RT_ENERGY_STATIC_MAX_GROUPS
 *   precision  RT_FP64 or RT_FP32_MIXED, the element type of U_dev
 *   cuda_stream  stream of the two kernel launches (NULL = legacy default stream)
 *   E_tot_dev  [G] DEVICE doubles receiving the sums, written asynchronously on the stream
 * The partial sums live in a fixed 32 KiB array in the library's device memory, held on
 * every GPU that loads the library until the process exits.  Each call overwrites the part
 * of it that it reads, so nothing carries over from the previous call, but calls that
 * overlap on the GPU share the array and race: order them on one stream.  The first call
 * on a device (and the first after the caller resets it) looks up the array's device address
 * with that device current; under CUDA's default lazy module loading that first call is also
 * when the library's code and this array are loaded onto the device.  So make one warm-up
 * call per device before a memory pool claims the whole GPU and before any stream capture.
 * Returns RT_ERR_INVALID for NULL pointers, n < 1, n_groups outside
 * [1, RT_ENERGY_STATIC_MAX_GROUPS] or an unknown precision; RT_ERR_CUDA if a CUDA call or a
 * launch fails, and also, before launching anything, when an error from the caller's earlier
 * CUDA work is still pending (it is left pending); there is no context, so no message. */
#define RT_ENERGY_STATIC_MAX_GROUPS 16
rt_status rt_energy_static(const void* U_dev, const double* V_dev, int64_t n, int32_t n_groups, int32_t precision,
                           void* cuda_stream, double* E_tot_dev);

/* Self-test of the bounded device waits (no paper counterpart): one warp waits, with the
 * wait of the pair kernels, on a shared-memory barrier that nothing completes, for
 * budget_cycles SM clock cycles (1 to 4e9), then records that the wait ran out.  Returns
 * RT_ERR_TIMEOUT when it did (the expected outcome) and RT_OK otherwise; the context stays
 * usable either way and its own time-out flag (rt_diag.wait_timeouts) is not touched.
 * Synchronises the context's stream; RT_ERR_INVALID for a budget outside the range. */
rt_status rt_wait_selftest(rt_ctx* ctx, uint64_t budget_cycles);

/* Per-particle geometry in caller order (device pointers, each may be NULL):
 * h [N], omega [N], V [N], B [N][3][3] (double). */
rt_status rt_particle_fields(rt_ctx* ctx, double* h_dev, double* omega_dev, double* V_dev, double* B_dev);

/* The symmetric neighbour lists in caller indices: offsets_dev [N+1] (int64),
 * cols_dev [n_directed] (int32); the order inside a row is the library's. */
rt_status rt_pairs(rt_ctx* ctx, int64_t* offsets_dev, int32_t* cols_dev);

/* Counters of the last rt_neighbours and of the steps since (host struct). */
rt_status rt_diagnostics(rt_ctx* ctx, rt_diag* out);

/* Per-kernel timing (tracing aid, no counterpart in the thesis).  With on = 1, later
 * rt_transport_step / rt_subcycle calls record CUDA events around every injection,
 * gradient, pair-flux and flux-gather launch (inside the captured graph as event nodes).
 * With on = k >= 2 they bracket the pair-flux launches only, one in every k - 1 of a call
 * (the first included; k = 2: all of them).  Each event pair serialises the graph around
 * its kernel: on the 262,144-particle set the 200 event nodes of on = 1 in a 50-sub-cycle
 * call add about 5% to it, the 100 of on = 2 about 2%.  0 turns it off.  Changing the
 * setting discards the captured graphs; RT_ERR_INVALID outside 0-1000. */
rt_status rt_set_profiling(rt_ctx* ctx, int32_t on);

/* Summed device time in milliseconds and number of launches per kernel kind
 * (ms_host[RT_KERNEL_KINDS], launches_host[RT_KERNEL_KINDS], host arrays) of the most
 * recent rt_transport_step or rt_subcycle call made with profiling on; zeros if none.
 * Synchronises the stream. */
rt_status rt_kernel_times(rt_ctx* ctx, double* ms_host, int64_t* launches_host);

/* HLL wave speeds (Eq. riemann-HLL): the largest (lmax_host) and smallest (lmin_host)
 * eigenvalue, in units of c, of the Jacobian of the M1 flux along a unit normal n, for a
 * state of reduced flux f = |F| / (cE) at angle theta between F and n; row-major host
 * arrays [RT_WAVE_NF][RT_WAVE_NTH] over the grid above.  The flux transport kernels
 * interpolate this table bilinearly.  The library derives it on the host, without a context
 * or a GPU: the Jacobian analytically (the F component normal to the (n, F) plane decouples
 * with eigenvalue b(f) f cos theta), the remaining 3 x 3 block's characteristic cubic solved
 * in extended precision and polished by Newton steps; at f = 1 (free streaming) every
 * eigenvalue equals cos theta.  RT_ERR_INVALID for NULL arrays. */
rt_status rt_wave_table(double* lmax_host, double* lmin_host);

/* Photo-ionisation sink of the photon groups (Eqs. dEdt-group, dFdt-group): every group
 * loses energy and flux at the rate c n_j sigma^N_gj summed over the absorbing species j.
 * rt_set_absorbers computes, on the context's stream, alpha_g = sum_j sigma_host[g][j]
 * n_dev[j] per particle from the caller's species number densities n_dev (n_species x N
 * doubles, caller order, read during the call) and cross sections sigma_host (host, G x
 * n_species doubles, in units consistent with n, c and dt).  From then on rt_transport_step,
 * rt_subcycle and rt_autotune called with alpha_dev == NULL apply the forward-Euler sink
 * U_g <- U_g max(0, 1 - c alpha_g dt) per group (a non-NULL alpha_dev applies its grey sink
 * instead); n_dev == NULL clears the absorbers.  rt_adjoint refuses contexts with absorbers
 * unless a grey alpha_dev is given.  Synchronises the stream.  RT_ERR_INVALID for
 * n_species outside [1, 8] or negative or non-finite cross sections. */
rt_status rt_set_absorbers(rt_ctx* ctx, int32_t n_species, const double* n_dev, const double* sigma_host);

/* Host helpers of the photo-ionisation sink (no context or GPU), CGS units, frequencies in
 * Hz.  Species j: 0 = H0, 1 = He0, 2 = He+.
 * rt_cross_section: sigma_j(E) in cm^2 at photon energy E_eV (eV), the fit of
 *   Eq. sigma-parametrizaiton with the parameters of Table tab:cross-sections, zero below the
 *   ionisation energy of the species (Eqs. nuIonHI, nuIonHeI, nuIonHeII).
 * rt_blackbody_groups: for a blackbody of temperature T_bb (Eq. blackbody) and groups
 *   [nu_edges[g], nu_edges[g+1]) (n_groups + 1 ascending edges; the last may be +inf), the
 *   mean photon energy eps_mean[g] (erg) and the number- and energy-weighted cross
 *   sections sigma_N[g][j], sigma_E[g][j] (cm^2, Eqs. sigma_N, sigma_E; host arrays G, G x 3).
 * rt_photon_number_to_luminosity: the group luminosities L_out[g] (erg/s) of a source
 *   emitting Ndot photons/s above nu_edges[0] with that spectrum (Appendix "Converting
 *   Photon Number Emission Rates to Photon Energy Emission Rates").
 * RT_ERR_INVALID for NULL arrays, non-positive temperatures or unordered edges. */
rt_status rt_cross_section(int32_t species, double E_eV, double* sigma_out);
rt_status rt_blackbody_groups(double T_bb, int32_t n_groups, const double* nu_edges, double* eps_mean,
                              double* sigma_N, double* sigma_E);
rt_status rt_photon_number_to_luminosity(double T_bb, double Ndot, int32_t n_groups, const double* nu_edges,
                                         double* L_out);

/* Set (rt_set_tuning) or read (rt_get_tuning) the launch variants of the float pair kernels
 * and the shapes above (host struct, copied).  RT_ERR_INVALID for a value outside those
 * listed; the context is unchanged then.  Valid before or after rt_neighbours. */
rt_status rt_set_tuning(rt_ctx* ctx, const rt_tuning* tuning);
rt_status rt_get_tuning(const rt_ctx* ctx, rt_tuning* tuning);

/* Number of launch-variant combinations rt_autotune tries: candidate k is
 * {flux_variant k / 6, gather_variant (k / 3) % 2, gradient_variant k % 3}, with the shapes
 * (cell_eighths ... pair_warps) of the context's current tuning. */
#define RT_TUNE_CANDIDATES 18

/* Autotuner (no paper counterpart): times n_sub plain transport steps of every candidate
 * launch-variant combination on the caller's state U_dev (4G x N, caller order, element
 * type per precision; read only) with luminosities Lsrc_dev (S x G or NULL) and absorption
 * alpha_dev (N or NULL), on the context's stream with CUDA events, keeping the fastest of
 * `repeats` repetitions (after one warm-up) per candidate; then adopts the fastest candidate
 * (as rt_set_tuning, dropping captured graphs) and returns it in *best (host struct).
 * ms_out (host, RT_TUNE_CANDIDATES doubles, may be NULL) receives each candidate's time.
 * The double path has one variant: every entry repeats the first.  Synchronises the
 * stream; uses the context's state buffers, so it must not overlap other calls on the
 * context.  RT_ERR_INVALID for n_sub outside [1, 1000] or repeats outside [1, 100]. */
rt_status rt_autotune(rt_ctx* ctx, const void* U_dev, double dt, int32_t n_sub, const double* Lsrc_dev,
                      const double* alpha_dev, int32_t repeats, rt_tuning* best, double* ms_out);

/* Message of the last failure ("" if none).  Valid until the next call on ctx. */
const char* rt_last_error(const rt_ctx* ctx);

/* Release everything the context owns (NULL is accepted). */
void rt_destroy(rt_ctx* ctx);

#ifdef __cplusplus
}
#endif

#endif /* RT_GB300_RT_H */
