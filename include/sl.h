/*
 * sl.h -- C ABI of the GB300 (sm_103a) semi-Lagrangian Monte-Carlo solver.
 *
 * The library advances N_s Monte-Carlo samples of a nodal polynomial field on
 * a periodic spectral-element mesh by the element-local semi-Lagrangian step
 * of Natarajan, Popov & Jacobs (arXiv:2009.07340, Section 5):
 *
 *   1. particles are seeded at the element's Chebyshev-Gauss nodes
 *      (Section 5.1, Eq. soln_init; nodes of Eq. gaussquad with (i+1/2)/N);
 *   2. they move by one explicit Euler-Maruyama step,
 *      x* = x + u(x) dt + sqrt(2 D(x)) dW^s, with ONE Wiener increment per
 *      sample, step and dimension shared by every node of every element
 *      (Section 5.2, Eq. def_dx and the paragraph after it), and the carried
 *      value gets the compositional update phi* = phi (1 - dt div u)
 *      (Eq. advection_phi);
 *   3. the advected interpolant (Eq. phi_stardef, Eq. h_star) is evaluated at
 *      the element faces (Eq. remap_bnd), an upwind value is taken at every
 *      interface (Eq. bnd_update), and the field is remapped to the Gauss
 *      nodes by the constrained least-squares fit
 *      q = argmin |V q - phi*|^2 + |B q - g|^2 (Section 5.3);
 *   4. samples are averaged on the nodes (Section 5.4, Eq. averaged).
 *
 * All arithmetic of these steps runs in the library's CUDA kernels.  The
 * Wiener increments come from Philox4x32-10 (Salmon et al., SC'11) with key
 * (seed low word, seed high word) and counter (step, sample, 0, 0), mapped to
 * two 52-bit uniforms u = (2x+1) 2^-53 and Box-Muller normals, so a given
 * (seed, step counter) fixes the result.
 *
 * Conventions
 *   - Node layout: element-major, elements x-fastest; inside an element the
 *     nodes are x-fastest (p = j*N + i in 2D).  Per-sample state is
 *     [sample][element][node].
 *   - Host pointers are caller-owned and only read/written during the call.
 *     "device" pointers are caller-owned CUDA device memory.
 *   - Every entry point returns SL_OK (0) or a negative SL_ERR_* code.  After
 *     SL_ERR_CUDA, SL_ERR_SINGULAR or SL_ERR_TIMEOUT the context is poisoned:
 *     only sl_free is valid.  Argument errors leave the context usable.
 *   - One context per host thread at a time; contexts are independent.
 */
#ifndef SL_H
#define SL_H

#include <stddef.h> /* size_t */

#ifdef __cplusplus
extern "C" {
#endif

enum {
    SL_OK = 0,
    SL_ERR_ARG = -1,         /* invalid argument (sizes, kinds, D < 0, NULL) */
    SL_ERR_DT = -2,          /* dt above the Eq. (1d_timestep) bound with strict_dt set */
    SL_ERR_OOM = -3,         /* device allocation failed */
    SL_ERR_CUDA = -4,        /* a CUDA call failed */
    SL_ERR_SINGULAR = -5,    /* coincident advected particles: non-finite remap */
    SL_ERR_TIMEOUT = -6,     /* a bounded device wait expired */
    SL_ERR_STATE = -7,       /* context poisoned by an earlier error */
    SL_ERR_UNSUPPORTED = -8  /* valid but not provided (e.g. 2D order above the limit) */
};

/* Arithmetic of the step.  Wiener increments and moments are FP64 always.  */
enum {
    SL_FP64 = 0,  /* everything in FP64                                       */
    SL_MIXED = 1, /* basis evaluation / remap contractions in FP32, the       */
                  /* constrained least-squares (capacitance) factor in FP64  */
                  /* (2D: the iterative remap's 4N x 4N capacitance matrix;  */
                  /* its direct fallback factors in FP32)                    */
    SL_FP32 = 2   /* as SL_MIXED but the factor in FP32 too                   */
};

/* Prescribed fields (all evaluated in physical coordinates).               */
enum {
    /* drift u */
    SL_U_CONST = 1,    /* u = (p0, p1)                                        */
    SL_U_SIN = 2,      /* u = p0 + p1 sin(p2 pi x)                       (1D) */
    SL_U_ROTATION = 3, /* u = p0 (-(y - p2), x - p1)                     (2D) */
    SL_U_NODAL = 4,    /* nodal: [dim][elements][N^dim] u_x (then u_y), see below */
    /* diffusion coefficient D >= 0 */
    SL_D_CONST = 11,   /* D = p0                                              */
    SL_D_COS = 12,     /* D = p0 (1 + p1 cos(p2 pi x))                        */
    SL_D_SINSIN = 13,  /* D = p0 (1 + p1 sin(p2 pi x) sin(p3 pi y))           */
    SL_D_NODAL = 14,   /* nodal: [elements][N^dim] D >= 0, see below           */
    /* initial condition phi0 */
    SL_PHI_GAUSS = 21,   /* p0 exp(-|x - (p2,p3)|^2 / (2 p1^2)), nearest periodic images */
    SL_PHI_FOURIER = 22, /* p0 + sum_{k=1}^{p2} a_k cos(k p1 pi x) + b_k sin(k p1 pi x), */
                         /* a_k = p[3+2(k-1)], b_k = p[4+2(k-1)], at most 18 modes (1D)  */
    SL_PHI_SINE = 23,    /* p0 + p1 sin(2 pi p2 x)                               (1D)    */
    SL_PHI_SINSIN = 24,  /* p0 + p1 sin(2 pi p2 x) sin(2 pi p2 y)                (2D)    */
    SL_PHI_NODAL = 25    /* host array nodal[element][node] of the initial values        */
};

/* Nodal drift and diffusion: the form in which a field solver hands its    */
/* velocity and diffusivity over (Section 5.2 takes du/dx from the DSEM      */
/* solver).  `nodal` holds the values at the Gauss nodes, element-major and  */
/* x-fastest as the state.  The divergence of the drift is the spectral      */
/* derivative of the nodal values in each element.  `face` (optional) holds  */
/* the normal drift component, or D, at the interface points:                */
/*   1D [K+1]: x = lo + f h, f = 0..K;                                       */
/*   2D the vertical interfaces [K1][K0+1][N] (x = lo + f h0, y at the Gauss */
/*      nodes of the element row), then the horizontal ones [K1+1][K0][N].   */
/* On a periodic mesh the last interface of a line is its first and that    */
/* entry is not read.  face = NULL: the mean of the traces of the two        */
/* neighbouring elements' interpolants at the point (the inside trace at a   */
/* Dirichlet boundary), D clipped at 0 there.  D must be >= 0 at every node  */
/* and every given interface point (SL_ERR_ARG).  Both arrays are host       */
/* memory, copied before the call returns.                                   */
typedef struct {
    int kind;
    double p[40];
    const double *nodal; /* *_NODAL kinds: host node values (SL_PHI_NODAL: [elements][N^dim]) */
    const double *face;  /* SL_U_NODAL / SL_D_NODAL: host interface table, or NULL            */
} sl_field;

/* Uniform tensor mesh of K[0] (x K[1]) elements on [lo, hi]. */
typedef struct {
    int dim;         /* 1 or 2                                       */
    int K[2];        /* elements per direction; K[1] ignored in 1D    */
    double lo[2];
    double hi[2];
    int periodic[2]; /* 1: periodic; 0: Dirichlet boundaries whose values the   */
                     /* caller gives per step with sl_set_boundary (2D: both 0)  */
} sl_mesh;

typedef struct {
    unsigned long long seed; /* Philox key                                           */
    int precision;           /* SL_FP64, SL_MIXED or SL_FP32                          */
    int strict_dt;           /* 1: sl_step refuses dt above the Eq. (1d_timestep) bound */
    void *stream;            /* cudaStream_t for all work; NULL = legacy default stream */
    int device;              /* CUDA device ordinal; -1 = current device              */
    long long sample0;       /* global index of sample 0 (Philox counter word 1): a run */
                             /* split over GPUs gives each a disjoint sample range;    */
                             /* sample0 + M <= 2^32                                     */
    double bc_weight;        /* weight w of the boundary rows of the remap,           */
                             /* min |V q - phi*|^2 + w^2 |B q - g|^2 (Section 5.3);   */
                             /* <= 0 means 1; INFINITY: the face values are hard     */
                             /* constraints, B q = g (1D only; SL_ERR_UNSUPPORTED in */
                             /* 2D); NaN: SL_ERR_ARG                                 */
    long long launch_chunk;  /* 2D: at most this many element-sample pairs per kernel  */
                             /* launch (0 = one launch per phase; results unchanged). */
                             /* Bounds how long one launch holds the GPU, so that     */
                             /* other streams' kernels start between launches.  When */
                             /* set, sl_step keeps at most 2 launches queued on the  */
                             /* stream, waiting on the host for earlier ones, and so */
                             /* returns only when the last launches are queued       */
    int components;          /* scalar fields per sample sharing the particles and    */
                             /* so the remap factorization (Section 5.3: its cost     */
                             /* does not grow with the components); 0 or 1: one; 2:   */
                             /* two (periodic meshes; 1D in SL_FP64 or SL_FP32, 2D   */
                             /* N <= 8 in any precision; otherwise                   */
                             /* SL_ERR_UNSUPPORTED).  Each sample's state, samples   */
                             /* and moments are [components][elements][N^dim]; every */
                             /* component starts from phi0 (set others with          */
                             /* sl_set_samples)                                       */
    int reseed_every;        /* > 0: after every step n with (n + 1) % reseed_every  */
                             /* == 0, every sample is set to the sample mean         */
                             /* (Eq. re-seed; the paper reseeds every 100 steps with  */
                             /* Dirichlet boundaries); 0: never                       */
} sl_options;

typedef struct sl_ctx sl_ctx; /* opaque; owns all of its device memory */

/* Prepares every kernel of the library on `device` (-1 = current device),  */
/* once per process: loads it and sets its shared-memory limit, and creates */
/* the library's memory pool for the device.  Under CUDA's lazy module      */
/* loading a kernel is loaded at its first launch, and a load may wait for  */
/* all work on the device; a solver created while other solvers' long       */
/* kernels run would then stall.  sl_init, sl_batch_create and              */
/* sl_server_create call it; calling it earlier moves the cost (tens of     */
/* milliseconds) to a time of the caller's choosing.  SL_OK or SL_ERR_CUDA. */
int sl_preload(int device);

/* Creates a solver for M samples of order N (N Gauss nodes per direction,  */
/* 2 <= N <= 16) on `mesh`, evaluates the fields at the nodes and faces and  */
/* sets every sample to phi0 (Section 5.1).  1D: K <= 2048 elements.         */
/* 2D: N <= 11 in SL_FP64, N <= 12 in the FP32 modes (SL_ERR_UNSUPPORTED     */
/* otherwise); in 2D both FP32 modes run the FP32 Gram solve with one         */
/* refinement step.                                                           */
/* The step counter starts at 0.  opt may be NULL (seed 0, SL_FP64).         */
int sl_init(sl_ctx **out, const sl_mesh *mesh, int N, int M, const sl_field *drift,
            const sl_field *diffusion, const sl_field *phi0, const sl_options *opt);

/* New drift and diffusion fields for the following steps (a time-dependent */
/* or externally computed flow, e.g. the velocity of an Eulerian solver the */
/* particles are coupled to): the node and face coefficients, the           */
/* divergence (spectral differentiation of the nodal drift) and the         */
/* time-step bounds are evaluated again; the samples are not touched.       */
/* Stream-ordered after earlier steps; synchronises the context's stream.   */
int sl_set_fields(sl_ctx *c, const sl_field *drift, const sl_field *diffusion);

/* As sl_set_fields for a field solver that runs on the same GPU: stream-     */
/* ordered on the context's stream, with no copy and no synchronisation.     */
/* The tables of SL_U_NODAL / SL_D_NODAL (same layouts) are DEVICE pointers,  */
/* read in place by kernels on the context's stream: they must hold their    */
/* values when those kernels run (e.g. written before on the same stream)    */
/* and stay allocated until then.  A D below 0 (or NaN) in a nodal table is  */
/* found on the device and reported as SL_ERR_ARG by the next synchronising  */
/* call (sl_moments, sl_get_samples), which poisons the context.  The time-  */
/* step bounds are recomputed when next needed (sl_dt_max, sl_dt_edge, or    */
/* sl_step with strict_dt), which synchronises then.                         */
int sl_set_fields_device(sl_ctx *c, const sl_field *drift, const sl_field *diffusion);

/* Dirichlet boundary values (1D, periodic[0] = 0), Section 5.3: at a domain */
/* boundary the given value is the ghost solution that takes the place of   */
/* the missing neighbour in the upwind rule (Eq. bnd_update).  values: host */
/* [nsteps][width], the values at the end of each of the next nsteps steps  */
/* (step counters n .. n + nsteps - 1 from the current one), copied before  */
/* return.  1D: width 2, the values at x = lo and x = hi.  2D: width        */
/* 2 (K[0] + K[1]) N, the face points of the left boundary x = lo ([K[1]][N], */
/* along y), the right boundary x = hi ([K[1]][N]), the bottom y = lo       */
/* ([K[0]][N], along x) and the top y = hi ([K[0]][N]), each at the Gauss   */
/* nodes of the boundary elements.  Each call replaces the previous table;  */
/* sl_step returns SL_ERR_ARG for a step the table does not cover.          */
/* SL_ERR_ARG on a periodic context.                                         */
int sl_set_boundary(sl_ctx *c, int nsteps, const double *values);

/* Sets every sample to the current sample mean (Eq. re-seed), on the       */
/* context's stream.  sl_step does this itself when reseed_every > 0.       */
int sl_reseed(sl_ctx *c);

/* Advances every sample by `steps` SL steps of size dt (Sections 5.2-5.3):  */
/* Wiener increments for the step counters [n, n+steps), particle advance,   */
/* face values, upwinding, constrained least-squares remap.  Asynchronous on */
/* the context's stream; the step counter advances by `steps`.  Returns      */
/* SL_ERR_DT if strict_dt is set and dt exceeds sl_dt_max.                   */
int sl_step(sl_ctx *c, double dt, int steps);

/* Sample moments on the nodes, Eq. (averaged): mean = (1/M) sum_s Q^s and   */
/* m2 = (1/M) sum_s (Q^s)^2, FP64 accumulation in a fixed order.  Host       */
/* arrays [elements][N^dim]; m2 may be NULL.  Synchronises the stream and    */
/* reports any deferred device error (SL_ERR_SINGULAR, SL_ERR_CUDA).         */
int sl_moments(sl_ctx *c, double *mean, double *m2);

/* As sl_moments into caller-owned device memory, asynchronously on the      */
/* context's stream (no synchronisation, no error check of earlier steps).  */
int sl_moments_device(sl_ctx *c, double *d_mean, double *d_m2);

/* Partial sums of the sample moments, for combining contexts that hold     */
/* disjoint sample ranges (one per GPU or process): the samples are          */
/* independent (Section 5.2: one Wiener increment per sample), so the moments */
/* of Eq. (averaged) over all of them are sums of per-range sums.            */
/*   d_psum  device, FP64 [nchunks][elements * N^dim (* components)]: row c    */
/*           = sum of the context's samples [64c, 64c + 64) (the last chunk   */
/*           may be shorter), in the same fixed order as sl_moments            */
/*   d_psq   device, FP64, same layout: sums of squares                       */
/* nchunks = ceil(M / 64) (sl_moment_chunk gives 64).  Caller-owned,          */
/* asynchronous on the context's stream.  Adding the chunk rows of all       */
/* contexts in ascending global sample order and dividing by the total       */
/* sample count reproduces sl_moments of one context holding every sample,  */
/* bit for bit, when every context's sample0 is a multiple of 64.            */
int sl_moments_partial(sl_ctx *c, double *d_psum, double *d_psq);

/* Samples per chunk of sl_moments_partial (64). */
int sl_moment_chunk(void);

/* Moments from chunk partial sums gathered from several contexts (the last */
/* pass of sl_moments): mean[v] = (sum_c psum[c][v]) / M_total and m2[v] =   */
/* (sum_c psq[c][v]) / M_total, the chunks added in ascending c, FP64.       */
/*   d_psum, d_psq  device [nchunks][V], caller-owned, read only             */
/*   d_mean         device [V]; d_m2 device [V] or NULL                       */
/*   stream         cudaStream_t or NULL; asynchronous on it                  */
/* SL_ERR_ARG for nchunks < 1, V < 1, M_total < 1 or a NULL input.           */
int sl_moments_combine(const double *d_psum, const double *d_psq, int nchunks, long long V, long long M_total,
                       double *d_mean, double *d_m2, void *stream);

/* The PDF at every node recovered by binning the samples (Section 5.4):    */
/* counts [elements][N^dim][nbins] (uint32) of the M samples in nbins equal */
/* bins over [lo, hi]: bin b = floor((x - lo) * (nbins / (hi - lo))) in    */
/* FP64 (FP32 pair states as hi + lo), x = hi in the last bin, x outside    */
/* [lo, hi] or NaN not counted.  1 <= nbins <= 4096, lo < hi finite.        */
/* sl_pdf: host counts, synchronous; sl_pdf_device: caller-owned device     */
/* counts, asynchronous on the context's stream.                            */
int sl_pdf(sl_ctx *c, int nbins, double lo, double hi, unsigned int *counts);
int sl_pdf_device(sl_ctx *c, int nbins, double lo, double hi, unsigned int *d_counts);

/* Largest dt satisfying |u|max dt + sqrt(2 Dmax dt) <= dx_min in every      */
/* direction (Eq. 1d_timestep), dx_min = smallest node gap times h.  In 2D   */
/* the step is not stable at this bound: a perturbation of the state grows  */
/* ~12 % per step there on 64x64 elements of N = 8 (measured on an FP64     */
/* reference); half of it is stable for a rotating drift, and a strong      */
/* uniform drift needs a quarter or less.  2D workloads take a fraction.    */
int sl_dt_max(const sl_ctx *c, double *dt);

/* The same bound with dx_min = the first Gauss node's distance to the       */
/* element face: at this dt a particle moved by u dt + one standard           */
/* deviation of the diffusion stays inside its element, the paper's reason  */
/* for restricting dt (Section 5.2: the interpolation matrix stays well      */
/* conditioned).  In 2D the remap solves with that matrix, so 2D workloads    */
/* use this bound: at the node-gap bound its condition number reaches ~3e3   */
/* at one standard deviation and ~5e7 at three (N = 8).                       */
int sl_dt_edge(const sl_ctx *c, double *dt);

/* Step counter (number of SL steps taken so far). */
int sl_step_count(const sl_ctx *c, long long *n);

/* 2D: how many element-sample groups the iterative (tensor-preconditioned)  */
/* solve handed to the direct solve since the context was created, per      */
/* phase: phase 1 = the interpolant's face values (Eq. remap_bnd), phase 2 = */
/* the constrained remap.  A group goes there when its conditioning test    */
/* fails or the iteration has not converged within its limit; the result   */
/* is the same solution either way.  Either pointer may be NULL.  1D        */
/* contexts report 0.  Synchronises; SL_ERR_ARG for a NULL context.         */
int sl_fallback_count(sl_ctx *c, long long *phase1, long long *phase2);

/* Copies samples [s0, s0+count) of the state to host memory, FP64,          */
/* [count][elements][N^dim].  Synchronises.                                   */
int sl_get_samples(sl_ctx *c, int s0, int count, double *out);

/* Overwrites samples [s0, s0+count) from host FP64 [count][elements][N^dim] */
/* (checkpoint restore together with sl_set_step_count).  Synchronises.    */
int sl_set_samples(sl_ctx *c, int s0, int count, const double *in);
int sl_set_step_count(sl_ctx *c, long long n);

/* Wiener increments dW for step counters [step0, step0+nsteps) and every    */
/* sample, computed by the device generator: host out[nsteps][M][dim].       */
int sl_wiener(sl_ctx *c, long long step0, int nsteps, double dt, double *out);

/* Kernel timing hook.  While enabled, sl_step records a pair of CUDA events */
/* on the context's stream around every launch of the step kernel (not the  */
/* Wiener-increment kernel).  sl_profile_read synchronises, returns the     */
/* summed event time (ms) and the number of such launches since the         */
/* previous read, and clears them.                                          */
int sl_profile(sl_ctx *c, int enable);
int sl_profile_read(sl_ctx *c, double *kernel_ms, long long *launches);

/* ------------------------------------------------------------------------ */
/* Batches: many independent solves of uneven size (mesh, N, M, dt, fields)  */
/* advanced together.  Each instance is a full solver (as sl_init); a call  */
/* of sl_batch_step advances all of them by `steps` steps of their own dt   */
/* with one CUDA-graph launch: a Wiener kernel over all instances, one       */
/* persistent kernel per 1D order (CTAs take (instance, sample-slot) work    */
/* items from an atomic counter; instances with K > 256 get their own        */
/* cluster launch), two launches per step per 2D order, and a step-counter   */
/* update.  The graph is captured on the first call with a given `steps`    */
/* and replayed afterwards.  Results per instance are the same as the        */
/* instance run alone with sl_init/sl_step (bitwise in SL_FP64).             */
/* ------------------------------------------------------------------------ */
typedef struct {
    sl_mesh mesh;
    int N, M;
    sl_field drift, diffusion, phi0;
    double dt;                /* dt_rule 0: the time step; 1: fraction of     */
                              /* sl_dt_max; 2: fraction of sl_dt_edge       */
    int dt_rule;
    unsigned long long seed;  /* this instance's Philox key                 */
    double bc_weight;         /* as sl_options.bc_weight                     */
} sl_instance;

typedef struct sl_batch sl_batch; /* opaque; owns its instances' device memory */

/* opt: precision, stream, device and strict_dt apply to every instance     */
/* (seed and sample0 are taken per instance).  A NULL stream makes the batch */
/* create its own non-blocking stream (graphs cannot be captured on the     */
/* legacy default stream).  Returns the first failing instance's error.    */
int sl_batch_create(sl_batch **out, int count, const sl_instance *inst, const sl_options *opt);

/* Advances every instance by `steps` steps (asynchronous on the stream).   */
int sl_batch_step(sl_batch *b, int steps);

/* Autotuner: for each 1D order, times the persistent kernel on the real    */
/* instances for `probe_steps` steps with 1..4 CTAs per SM and keeps the     */
/* fastest; then times whole steps with the order classes spread over 1, 2  */
/* or 4 parallel graph branches and keeps the fastest.  Every instance's    */
/* state and step counter are restored afterwards.  best_ms (may be NULL)  */
/* receives the best whole-step probe time.                                  */
int sl_batch_tune(sl_batch *b, int probe_steps, double *best_ms);

/* Persistent grid chosen for 1D class `cls` (order N, CTAs, instances).     */
int sl_batch_grid(const sl_batch *b, int cls, int *N, int *grid, int *instances);

/* Parallel graph branches a step's order classes are spread over (1 until  */
/* sl_batch_tune chooses).                                                   */
int sl_batch_lanes(const sl_batch *b, int *lanes);

/* Moments / samples of instance i (as sl_moments / sl_get_samples).         */
int sl_batch_moments(sl_batch *b, int i, double *mean, double *m2);
int sl_batch_samples(sl_batch *b, int i, int s0, int count, double *out);

void sl_batch_free(sl_batch *b);

/* ------------------------------------------------------------------------ */
/* Serving: solves submitted over time, run with continuous batching.  A     */
/* scheduler thread admits queued requests in arrival order, backfilling,    */
/* while their device footprint fits in `budget_bytes` beside the running    */
/* ones (a request larger than the budget is rejected with SL_ERR_OOM).     */
/* Light requests (up to ~2e9 operations per step) run on high-priority     */
/* streams by slices of up to `slice_steps` steps; a host callback at the    */
/* end of each slice hands the request back to the scheduler for the next   */
/* one, so requests' kernels overlap on the GPU.  A heavy request runs on a  */
/* low-priority stream, driven by a worker thread of its own one step at a  */
/* time in short launches with a bounded queue (sl_options.launch_chunk),   */
/* so that it never holds the GPU or a hardware queue for long.  Solvers    */
/* are created and completed (moments, memory released, latency =          */
/* completion minus submission) on worker threads.  Each result equals the  */
/* request run alone.                                                       */
/* ------------------------------------------------------------------------ */
typedef struct {
    size_t budget_bytes; /* device memory the running requests may hold;      */
                         /* reserved when the server is created (SL_ERR_OOM  */
                         /* if the device cannot hold it)                    */
    int slice_steps;     /* steps per request per scheduling round (>= 1)      */
    int heavy_slots;     /* heavy requests (estimated >= ~1 ms of GPU work per  */
                         /* step) running at once, each driven by a worker     */
                         /* thread of its own; 0 = admitted by the budget      */
                         /* alone and served by 2 threads in arrival order     */
    int precision;       /* SL_FP64, SL_MIXED or SL_FP32                        */
    int device;          /* CUDA device ordinal; -1 = current                   */
    int max_active;      /* requests admitted and not finished at once; 0 = no  */
                         /* limit (the budget and heavy_slots alone)            */
} sl_server_config;

typedef struct {
    long long submitted, completed, rejected, failed, running, queued;
    long long esu_completed;            /* element-sample updates of completed requests */
    long long memory_in_use, memory_peak;
    double p50_s, p99_s, mean_s;        /* latency of completed requests             */
    double span_s;                      /* first submission to last completion       */
    double esu_per_s;                   /* esu_completed / span_s                    */
    long long slices;                   /* light-request slices launched              */
    double sched_busy_s;                /* scheduler thread time spent working        */
    double launch_s, launch_max_s;      /* time in slice launches: total, longest     */
} sl_server_stats;

typedef struct sl_server sl_server;

int sl_server_create(sl_server **out, const sl_server_config *cfg);
/* Queues a request of `steps` steps of spec->dt; *ticket identifies it.    */
int sl_server_submit(sl_server *s, const sl_instance *spec, int steps, long long *ticket);
/* state: 0 queued, 1 running, 2 done, < 0 error code.  When done, copies   */
/* the moments (host [elements][N^dim]; either may be NULL) and latency.    */
int sl_server_poll(sl_server *s, long long ticket, int *state, double *mean, double *m2, double *latency_s);
/* Phases of a completed request, in seconds (out[9]):                     */
/*   out[0] queued: submission to admission (budget, slots)                */
/*   out[1] admission to the start of solver creation (worker wait)       */
/*   out[2] solver creation (stream, sl_init)                              */
/*   out[3] running: solver ready to its last slice seen complete          */
/*   out[4] last slice seen complete to the start of completion (wait)    */
/*   out[5] moments (computed and copied to the host)                      */
/*   out[6] release (solver, stream)                                       */
/*   out[7] total latency (the sum of out[0..6])                           */
/*   out[8] the longest slice turnaround (launch to completion seen)       */
/* SL_ERR_STATE if the request is not done.                                */
int sl_server_timing(sl_server *s, long long ticket, double *out);
/* Waits until nothing is queued or running (SL_ERR_TIMEOUT after timeout_s). */
int sl_server_wait_idle(sl_server *s, double timeout_s);
int sl_server_stats_get(sl_server *s, sl_server_stats *out);
/* Stops: slices in flight complete, queued and running requests are        */
/* abandoned, everything is released.                                        */
void sl_server_free(sl_server *s);

/* Allocation-free sample moments.  The paper has no counterpart: this entry  */
/* exists for callers that cannot call cudaMalloc when they need the moments */
/* (a serving loop whose HBM budget is fully reserved up front, code that     */
/* must not let an allocation synchronise the device, a host framework that   */
/* owns all device memory through its own pool).  No context is needed.     */
/*   d_samples  device, FP64 [M][V] (sample-major), caller-owned, read only   */
/*   d_mean     device, FP64 [V]: (1/M) sum_s samples[s][v]                   */
/*   d_m2       device, FP64 [V] or NULL: (1/M) sum_s samples[s][v]^2         */
/*   stream     cudaStream_t or NULL; the call is asynchronous on it          */
/* Partial sums go to one fixed device array of 2^21 doubles (16 MiB) that    */
/* every GPU loading the library holds until exit; hence V <= 2^20 nodes      */
/* (larger V returns SL_ERR_ARG), and no cudaMalloc, cudaFree or allocating   */
/* library routine is called.  The first call on a device looks up the        */
/* array's device address (once per device); make that first call before any */
/* stream capture.  All calls on a device share the array: calls that may    */
/* overlap on the GPU (different streams without ordering) race and give     */
/* wrong results.  Each call writes every partial it reads, so no clearing   */
/* is needed between calls.                                                   */
int sl_moments_static(const double *d_samples, int M, long long V, double *d_mean, double *d_m2,
                      void *stream);

/* Releases the context and its device memory.  NULL is a no-op. */
void sl_free(sl_ctx *c);

/* Static string describing an SL_* code. */
const char *sl_strerror(int code);

#ifdef __cplusplus
}
#endif
#endif /* SL_H */
