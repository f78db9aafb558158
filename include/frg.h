/*
 * frg.h -- C ABI of the GB300 (sm_103a) one-loop fRG library.
 *
 * The problem (the paper, Sec. 2, Eq. 1): an ODE dV/dg = F[V; g] for one flat
 * array V of discretised correlation functions, integrated with an explicit
 * stepper so that every component of F can be computed independently at fixed
 * V; the right-hand side is a numerical treatment of three one-loop diagrams
 * (Sec. 4); the flow of the self-energy is the extension named in Sec. 2.
 *
 * The instance implemented here is the single-impurity Anderson model in
 * Matsubara frequencies with the Omega-scheme cutoff:
 *   G0^{-1}(iw) = iw - (eps_d + U/2) + i Delta sgn(w)     (Hartree U/2 absorbed)
 *   G_L = 1/(Theta^{-1} G0^{-1} - Sigma),   Theta_L(w) = w^2/(w^2 + L^2)
 *   S_L = -G^2 (2L/w^2) G0^{-1},            Lb(a,b) = S(a)G(b) + G(a)S(b)
 * State per parameter point: the up-down vertex V(k1,k2,k3) on an N x N x N box
 * of fermionic Matsubara indices and the self-energy Sigma on N frequencies.
 * Flow variable l = ln L, from L0 down to L_f:
 *   dV/dl = L (Tpp + Tdph + Txph)                 (three one-loop channels)
 *   Tpp  = -T sum_p V(k1,k2,p) Lb(p,s-p) V(p,s-p,k3),                s = k1+k2
 *   Tdph = +T sum_p Lb(p,p-t) [2V(k1,p,k3)V(p-t,k2,p) - V(k1,p,p-t)V(p-t,k2,p)
 *                              - V(k1,p,k3)V(p-t,k2,k4)],           t = k3-k1
 *   Txph = -T sum_p V(k1,p+Q,p) Lb(p,p+Q) V(p,k2,k3),                Q = k2-k3
 *   dSigma(w)/dl = L T sum_p S(p) [2V(w,p,w) - V(w,p,p)]
 * V takes the stored value when all four frequencies lie in the box and the
 * bare U otherwise; loop sums run over internal frequencies inside the box.
 *
 * Memory conventions (all calls):
 *  - Vertex buffers: N^3 complex128, interleaved (re, im), index
 *    ((i1*N)+i2)*N+i3 with i = n + N/2 for Matsubara index n in [-N/2, N/2).
 *    Self-energy buffers: N complex128.
 *  - "d_" pointers are device pointers on the context's device, "h_" pointers
 *    host pointers (pageable or pinned).  Buffers passed in stay owned by the
 *    caller; the context owns its state and workspace.
 *  - Work is issued on the stream given at frg_init (0 = legacy default
 *    stream); calls that return results to host memory synchronise it.
 *  - Every call returns FRG_OK (0) or a negative FRG_E* code; no exception or
 *    abort crosses the ABI.  frg_last_error() describes the last failure.
 *  - One context per host thread at a time.
 */
#ifndef FRG_H
#define FRG_H

#ifdef __cplusplus
extern "C" {
#endif

#define FRG_OK 0
#define FRG_EINVAL (-1)      /* bad argument or parameter */
#define FRG_ENOMEM (-2)      /* device or host allocation failed */
#define FRG_ECUDA (-3)       /* a CUDA call failed */
#define FRG_ENONFINITE (-4)  /* NaN/Inf in the state or the error norm */
#define FRG_ENOTCONV (-5)    /* step size underflow or step limit reached */
#define FRG_ETIMEOUT (-6)    /* a bounded device-side wait ran out */

/*
 * Arithmetic of the channel contractions.  Every precision evaluates the three
 * channel sums above for whatever vertex it is given: each operand is read as
 * the entry the sum names (no crossing, reversal or particle-hole symmetry of
 * V is assumed; only FRG_REVERSAL below is an assertion about the inputs).
 * The split precisions differ from FP64 by rounding alone: the vertex is
 * rounded to FP32 and the products run on the tensor cores (normwise relative
 * error of one rhs below 1e-6 for FRG_3XTF32 and 5e-5 for FRG_BF16X3 on the
 * test inputs; whole flows within 1e-6 of the FP64 oracle).
 */
#define FRG_FP64 0    /* everything in FP64 (CUDA cores) */
#define FRG_3XTF32 1  /* split-TF32 (hi*hi + hi*lo + lo*hi) on tcgen05, FP32 accumulate */
#define FRG_BF16X3 2  /* three BF16 slices, six products, on tcgen05, FP32 accumulate */

/* channel_mask bits */
#define FRG_CH_PP 0x1
#define FRG_CH_DPH 0x2
#define FRG_CH_XPH 0x4
#define FRG_CH_SIGMA 0x8
#define FRG_CH_ALL 0xF
/*
 * Frequency-box tails (an option beyond the paper's box truncation): the
 * internal sum of every enabled channel and of the self-energy runs over a
 * window of FRG_TAIL_FACTOR * N_f Matsubara indices centred on the box
 * (both internal frequencies in the window) instead of the box.  Vertices keep
 * the box rule (bare U as soon as an index leaves the box) and the propagators
 * outside the box take Sigma = 0.  Every vertex with an internal index
 * outside the box is then U, so the extra terms are -Lambda T U^2 times a
 * bubble sum per transfer for pp (s = k1 + k2) and xph (Q = k2 - k3), zero for
 * the direct particle-hole channel, and Lambda T U sum S for the self-energy;
 * the library evaluates them in FP64 per rhs.  frg_rhs_noalloc rejects the
 * bit (FRG_EINVAL).
 */
#define FRG_TAILS 0x10
#define FRG_TAIL_FACTOR 16
/*
 * Frequency-reversal reduction (split precisions; FRG_FP64 computes every
 * transfer whatever the bits).  A reversal-symmetric state,
 *   V(N-1-i1, N-1-i2, N-1-i3) = conj V(i1, i2, i3),  Sigma(N-1-i) = conj Sigma(i)
 * (index i = n + N/2, i.e. n -> -n-1 with complex conjugation), has a
 * reversal-symmetric rhs, channel by channel, and every flow from the bare
 * vertex keeps that symmetry exactly; the paper reduces its ODE system to the
 * independent couplings the same way (Sec. 4).  By default a split-precision
 * context uses the reduction for its flows (frg_flow, frg_advance) while the
 * state of every point is reversal-symmetric: always from frg_init, and
 * frg_set_state checks a new state exactly (entry by entry) and switches the
 * context's flows to computing every transfer while any point's state is
 * not.  frg_rhs then computes every transfer (its inputs are arbitrary).
 * FRG_NO_REVERSAL turns the reduction off; FRG_REVERSAL asserts instead that
 * every vertex and self-energy handed to the context, frg_rhs's included, is
 * reversal-symmetric, and halves the flow's storage (below).
 * With FRG_REVERSAL the caller asserts that every vertex and
 * self-energy handed to the context is reversal-symmetric,
 *   V(N-1-i1, N-1-i2, N-1-i3) = conj V(i1, i2, i3),  Sigma(N-1-i) = conj Sigma(i)
 * (index i = n + N/2, i.e. n -> -n-1 with complex conjugation), which every
 * flow from the bare vertex keeps exactly.  The rhs then has the same symmetry
 * channel by channel, transfer m of each channel (m = s, t + N - 1 or Q + N - 1)
 * mapping to 2N - 2 - m: the contraction computes the transfers m <= N - 1
 * only (about half of the tensor-core work) and the scatter-add takes the
 * others from the mirrored entries.  For inputs without the symmetry the
 * result is the symmetric part's rhs, not the input's.  In a flow the split
 * precisions also store half of the vertex: the stage derivatives and the
 * float-pair copy of the state hold the entries with i1 < N/2 only, the stage
 * sums and the error norm run over those, and every other entry of the state
 * is written as the conjugate of its mirror (so a state set with
 * frg_set_state enters the flow through its entries with i1 < N/2).
 * frg_rhs_noalloc rejects the bit (FRG_EINVAL).
 */
#define FRG_REVERSAL 0x20
#define FRG_NO_REVERSAL 0x40
/* Crossing reduction of the split-precision channel products (channel_mask
 * bit, paper Sec. 4: the reduction of the ODE system to independent couplings
 * by the model's symmetries).  With FRG_CROSSING the caller asserts that every
 * vertex handed to the context, frg_rhs's included, is crossing-symmetric,
 *   V(i1, i2, i3) = V(i2, i1, i4),  i4 = i1 + i2 - i3
 * (exchange of the two incoming and of the two outgoing particles), which the
 * flow from the bare vertex has in exact arithmetic.  Each channel's product
 * at a transfer m then holds pairs of equal entries: pp (s = m) the entries
 * (k1, k3) and (s - k1, s - k3); composed with the frequency reversal above,
 * which maps m to itself, the direct and the crossed channel the entries
 * (k1, k2) and (N-1-k2, N-1-k1), resp. (k3, k1) and (N-1-Q-k1, N-1-Q-k3), with
 * conjugate values.  Wherever the reversal reduction computes the transfers
 * m <= N - 1 (split precisions), the tiles of a transfer with more than 64
 * valid rows then skip one rectangle of such partners and write it from the
 * entries they computed (N <= 128 with one column tile of N columns; larger
 * grids compute every entry).  The flow's states are crossing-symmetric up to
 * the rounding of the split products, which is also the size of the change.
 * For inputs without the symmetry the result is not the input's rhs.  The FP64
 * path computes every entry; frg_rhs_noalloc rejects the bit (FRG_EINVAL). */
#define FRG_CROSSING 0x80

/*
 * Cutoff schemes (frg_params.cutoff).  Both regularise the bare propagator as
 * G0_L = Theta_L G0 and flow in l = ln Lambda from Lambda0 down to Lambda_f:
 *   FRG_CUTOFF_OMEGA        Theta = w^2 / (w^2 + Lambda^2); Lambda_f -> 0 is
 *                           the full model.
 *   FRG_CUTOFF_INTERACTION  the interaction flow: Theta = 1 / sqrt(Lambda),
 *                           i.e. G0_g = sqrt(g) G0 with g = 1 / Lambda, so that
 *                           the model at Lambda has the interaction U / Lambda
 *                           (after rescaling); Lambda = 1 (g = 1) is the full
 *                           model, Lambda0 = 1 / g0 >> 1 the start at V = U,
 *                           Sigma = 0.
 */
#define FRG_CUTOFF_OMEGA 0
#define FRG_CUTOFF_INTERACTION 1

typedef struct {
    double U;         /* interaction */
    double T;         /* temperature (> 0) */
    double eps_d;     /* level energy; particle-hole symmetry at eps_d = -U/2 */
    double Delta;     /* wide-band hybridisation (> 0) */
    int N_f;          /* fermionic frequencies per axis: even, 2 <= N_f <= 256 */
    double Lambda0;   /* initial scale (> Lambda_f > 0) */
    double Lambda_f;  /* final scale */
    double rtol;      /* relative tolerance of the step controller (> 0) */
    double atol;      /* absolute tolerance (>= 0) */
    double h0;        /* first step in l = ln Lambda (< 0); 0 selects -0.01 */
    long max_steps;   /* step attempts before FRG_ENOTCONV; 0 selects 100000 */
    int precision;    /* FRG_FP64, FRG_3XTF32 or FRG_BF16X3 */
    int channel_mask; /* FRG_CH_* bits, optionally | FRG_TAILS | FRG_REVERSAL or FRG_NO_REVERSAL | FRG_CROSSING; 0 selects FRG_CH_ALL */
    int cutoff;       /* FRG_CUTOFF_OMEGA (default) or FRG_CUTOFF_INTERACTION */
} frg_params;

typedef struct frg_ctx frg_ctx;

typedef struct {
    double Lambda;   /* scale reached */
    double h;        /* next step proposal in l */
    long accepted;   /* accepted steps */
    long rejected;   /* rejected steps */
    long rhs_evals;  /* right-hand-side evaluations */
    int status;      /* FRG_OK while running or done, else FRG_E* */
    int done;        /* 1 once Lambda_f is reached or the point failed */
} frg_flow_stats;

typedef struct {
    double sigma_lowest_re, sigma_lowest_im; /* Sigma(i pi T) */
    double Z;                                /* 1 / (1 - Im Sigma(i pi T) / (pi T)) */
    double U_eff_re, U_eff_im;               /* V at n1 = n2 = n3 = 0 */
    double n;                                /* 1/2 + T sum_box Re G (informational) */
} frg_obs;

/*
 * Create a context for n_points parameter points (params[0..n_points-1]): the
 * state of the paper's ODE (Sec. 2, Eq. 1) for each point, V and Sigma at the
 * initial scale, and the workspace of its right-hand side (Sec. 4).  All
 * points must share precision and channel_mask.  Allocates the device state
 * (initialised to V = U, Sigma = 0 at Lambda0) and all workspace, on the
 * current device.  cuda_stream is a cudaStream_t (may be NULL).
 * Errors: FRG_EINVAL (N_f odd or out of range, T <= 0, Delta <= 0, rtol <= 0,
 * Lambda_f >= Lambda0, mixed precision/mask, n_points < 1), FRG_ENOMEM,
 * FRG_ECUDA.  On error *out is NULL.
 */
int frg_init(const frg_params *params, int n_points, void *cuda_stream, frg_ctx **out);

/* Release everything the context owns.  NULL is ignored. */
void frg_destroy(frg_ctx *ctx);

/* Text of the last error on this context (never NULL). */
const char *frg_last_error(const frg_ctx *ctx);

/*
 * One evaluation of the right-hand side F[V; g] of the paper's ODE (Sec. 2,
 * Eq. 1; the three one-loop diagrams of Sec. 4 and the self-energy flow), i.e.
 * d/dl of (V, Sigma) as written at the top of this file, for point `point` at
 * scale Lambda (> 0), in the context's precision and channel mask: reads
 * d_gamma (N^3 complex128) and d_sigma (N complex128), writes d_dgamma and
 * d_dsigma (same shapes).  Any vertex is accepted (no symmetry is assumed,
 * unless the context was created with FRG_REVERSAL).  Device pointers,
 * caller-owned; asynchronous on the context stream.  d_sigma may be NULL
 * (Sigma = 0).  Uses the context workspace, so calls on one context must not
 * overlap.  Errors: FRG_EINVAL (point out of range, Lambda <= 0, NULL output
 * or d_gamma), FRG_ENOMEM (first call's scratch), FRG_ECUDA.
 */
int frg_rhs(frg_ctx *ctx, int point, double Lambda, const void *d_gamma,
            const void *d_sigma, void *d_dgamma, void *d_dsigma);

/*
 * Same as frg_rhs (paper Sec. 2, Eq. 1) with host buffers: copies the inputs to
 * the device, evaluates, copies the results back and synchronises the stream
 * before returning.
 */
int frg_rhs_host(frg_ctx *ctx, int point, double Lambda, const double *h_gamma,
                 const double *h_sigma, double *h_dgamma, double *h_dsigma);

/*
 * Pipelined host-buffer evaluations (paper Sec. 2, Eq. 1, as frg_rhs).  frg_rhs_host_async enqueues the same
 * evaluation as frg_rhs_host and returns at once: the host->device copy of the
 * input runs on a copy-in stream, the evaluation on the context stream, the
 * device->host copy of the result on a copy-out stream, through two device
 * buffer slots, so that in a sequence of calls the input of one evaluation, the
 * computation of the previous one and the output of the one before that overlap
 * (both directions of the host link busy at once).  The host buffers of a call
 * must stay valid, and the output buffers unread, until frg_sync returns; the
 * output buffers of calls in flight must not overlap.  frg_sync waits for every
 * enqueued evaluation and returns its first device-side failure
 * (FRG_ETIMEOUT); argument errors are returned by frg_rhs_host_async itself.
 */
int frg_rhs_host_async(frg_ctx *ctx, int point, double Lambda, const double *h_gamma,
                       const double *h_sigma, double *h_dgamma, double *h_dsigma);
int frg_sync(frg_ctx *ctx);

/*
 * Integrate the paper's ODE (Sec. 2, Eq. 1: an explicit stepper; Sec. 4: seven
 * rhs evaluations for the first step) for every point from its current state
 * to its Lambda_f with the Dormand-Prince 5(4) pair: device-resident stage
 * sums, embedded error norm and step control, one captured CUDA graph per step
 * attempt of all points.  stats (host, n_points entries, may be NULL) receives
 * the per-point statistics.  Returns FRG_OK if every point reached Lambda_f,
 * else the first failing point's code (FRG_ENONFINITE, FRG_ENOTCONV), or
 * FRG_ETIMEOUT / FRG_ECUDA.
 */
int frg_flow(frg_ctx *ctx, frg_flow_stats *stats);

/*
 * Advance every unfinished point by at most max_attempts step attempts
 * (accepted or rejected; the stepper of frg_flow, paper Sec. 2); finished
 * points are left alone.  Same error rules
 * as frg_flow.  Used for checkpointing and for timing a fixed amount of work.
 */
int frg_advance(frg_ctx *ctx, long max_attempts, frg_flow_stats *stats);

/*
 * Observables of point `point` at its current scale (synchronises).  The paper
 * names none for this model; these are the model's standard read-outs:
 * Sigma(i pi T), the quasiparticle weight Z = 1/(1 - Im Sigma(i pi T)/(pi T)),
 * the effective interaction U_eff = V at n1 = n2 = n3 = 0 (all four external
 * frequencies pi T) and the in-box occupation (informational).
 */
int frg_observables(frg_ctx *ctx, int point, frg_obs *out);

/*
 * Copy the current state (the ODE's V and Sigma, paper Sec. 2) of point
 * `point` out to caller device buffers
 * (d_gamma N^3, d_sigma N complex128), and its scale and next step (host).
 * Any of the output pointers may be NULL.  Synchronises.
 */
int frg_get_state(frg_ctx *ctx, int point, void *d_gamma, void *d_sigma,
                  double *Lambda, double *h);

/*
 * Replace the state (the ODE's V and Sigma, paper Sec. 2) of point `point`
 * (resume from a checkpoint or start from a custom state): device buffers
 * d_gamma / d_sigma (NULL sigma = 0), scale Lambda (Lambda_f < Lambda <=
 * Lambda0 is not required, but Lambda > Lambda_f for the point to flow) and
 * next step h in l (< 0; 0 selects the h0 of frg_init).  Any vertex is
 * accepted: by default a split-precision context checks the state's
 * reversal symmetry exactly and its flows use the reduction only while every
 * point's state has it; with FRG_REVERSAL the state enters through its entries
 * with i1 < N/2 (see there).  Clears the point's statistics and done flag.
 */
int frg_set_state(frg_ctx *ctx, int point, const void *d_gamma, const void *d_sigma,
                  double Lambda, double h);

/* Per-point statistics without advancing (synchronises). */
int frg_stats(frg_ctx *ctx, frg_flow_stats *stats);

/*
 * Diagnostics.  frg_rhs_timed evaluates exactly like frg_rhs and records CUDA
 * events on the context stream around its phases; ms[0..4] (host) receive the
 * durations of the bubble-weight (with the self-energy, which the same kernel
 * computes), operand-regather, channel-contraction and combine (scatter-add)
 * phases, and ms[4] the addition of the frequency-box tails (FRG_TAILS; 0
 * without them); 0 for a phase the path does not have.  Synchronises.
 * frg_kernel_launches returns the number of kernels this library has launched
 * in the process so far.
 */
int frg_rhs_timed(frg_ctx *ctx, int point, double Lambda, const void *d_gamma,
                  const void *d_sigma, void *d_dgamma, void *d_dsigma, float *ms);
long frg_kernel_launches(void);
/*
 * Tile geometry of the crossing reduction (diagnostic; FRG_CROSSING, paper
 * Sec. 4 symmetry reduction): for channel ch (0 pp, 1 direct, 2 crossed
 * particle-hole) at a transfer m <= N - 1 with more than 64 valid rows, on a
 * grid of N frequencies with tiles of nt columns (N <= nt <= 128, nt a multiple
 * of 16), row tile rt (0 or 1) computes the columns [out[0], out[0] + out[1])
 * (out[1] = 0: the tile is dropped), writes its own entries of the columns
 * [out[2], out[3]), and writes the crossing partners of its entries whose
 * column lies in [out[4], out[5]) and whose row (counted from the transfer's
 * first valid row) is at most out[6].  No device work.  Returns FRG_OK, or
 * FRG_EINVAL (arguments outside those ranges, out NULL).
 */
int frg_cross_tile(int ch, int N, int nt, int m, int rt, int out[7]);
/*
 * Failure-path self-test (no counterpart in the paper).  Every wait of the
 * tensor-core pipeline is bounded: a wait that runs out records the failure in
 * the context's device error word and the kernel returns, so the host sees
 * FRG_ETIMEOUT instead of a hung device.  frg_selftest_wait runs one such wait,
 * with a limit of limit_ms (clamped to [1, 2000] ms), on a barrier that nothing
 * completes, on the context stream; it returns FRG_ETIMEOUT when the mechanism
 * works (the error word is cleared again and the context stays usable), or
 * FRG_EINVAL / FRG_ECUDA.  Synchronises.
 */
int frg_selftest_wait(frg_ctx *ctx, double limit_ms);

/*
 * Contraction autotuning (split precisions).  The paper distributes work over
 * MPI ranks and has no tile shapes to tune; on this GPU the channel products
 * run as tiles of 64 complex rows x NT complex columns on persistent CTAs, and
 * the fastest NT and work assignment depend on the grid sizes of the batch.
 * frg_autotune times one rhs evaluation of every point of the context (at the
 * current flow state) for each candidate plan -- cap on NT of 128, 64 or 32
 * (NT = min(cap, N rounded up to 16)) times an epilogue allowance of 0, 3 or 8
 * k-steps per tile in the longest-first scheduler's cost model -- and keeps the
 * fastest plan for all later evaluations of the context.  Plans differ only in
 * how the same per-element sums are distributed, not in their arithmetic.
 * *out (may be NULL) receives the choice; an FP64 context has nothing to tune
 * (returns FRG_OK, out->candidates = 0).  Synchronises.
 */
typedef struct {
  int nt_cap;       /* chosen cap on the complex columns of a tile */
  int epi_cost;     /* chosen per-tile epilogue allowance (k-steps) */
  int candidates;   /* plans timed */
  float ms;         /* one rhs of all points with the chosen plan */
  float ms_default; /* the same with the default plan (128, 3) */
} frg_tune;
int frg_autotune(frg_ctx *ctx, frg_tune *out);

/*
 * Right-hand side without any device allocation (the paper has no counterpart;
 * this is a service for callers).  Some callers cannot allocate device memory
 * when they need an evaluation: a latency-critical loop in which an allocation
 * could stall or synchronise the device, or a process whose device memory is
 * owned by another component (a framework's caching allocator, a fixed memory
 * budget).  frg_rhs_noalloc needs no context: it evaluates d/dl of (V, Sigma)
 * for the single point *p at scale Lambda in FP64 (p->precision, Lambda0,
 * Lambda_f, tolerances and step settings are ignored; channel_mask applies),
 * reading d_gamma (N^3 complex128) and d_sigma (N complex128, may be NULL) and
 * writing d_dgamma and d_dsigma, all device pointers on the current device,
 * asynchronously on cuda_stream (a cudaStream_t, NULL for the legacy stream).
 * It calls no cudaMalloc, cudaFree or other allocating routine: its whole
 * workspace is one file-scope device array of about 290 KB that every GPU
 * which loads this library holds until the process exits.
 *  - Limit: N_f <= FRG_NOALLOC_MAX_N (even, >= 2); larger sizes, T <= 0,
 *    Delta <= 0, Lambda <= 0, non-finite parameters, NULL output pointers, or
 *    a channel_mask with FRG_TAILS, FRG_REVERSAL, FRG_NO_REVERSAL or
 *    FRG_CROSSING (anything above FRG_CH_ALL) return FRG_EINVAL without
 *    touching the device.
 *  - The first call on a device looks up the array's device address
 *    (cudaGetSymbolAddress) and caches it with the device's current context;
 *    the first call after that context changed (cudaDeviceReset, or another
 *    context made current) looks it up again.  Make such a first call before
 *    any stream capture on that device.
 *  - Every call on a device shares the array and leaves its contents behind;
 *    each call rewrites everything it reads.  Calls that overlap on the GPU
 *    (for example on two streams) race on the array: serialise them.
 * Returns FRG_OK, FRG_EINVAL or FRG_ECUDA (launch failure).
 */
#define FRG_NOALLOC_MAX_N 64
int frg_rhs_noalloc(const frg_params *p, double Lambda, const void *d_gamma,
                    const void *d_sigma, void *d_dgamma, void *d_dsigma,
                    void *cuda_stream);

#ifdef __cplusplus
}
#endif
#endif /* FRG_H */
