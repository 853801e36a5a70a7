/*
 * tdmix — time-dependent four-body amplitude likelihood on one GPU.
 *
 * C ABI of the library that evaluates the unbinned negative log-likelihood
 * (NLL) of D0 -> K+ pi- pi+ pi- decay events and its gradient, as described
 * in arXiv:1702.06735 (time-dependent amplitude analysis of a pseudoscalar
 * decaying to four pseudoscalars):
 *
 *   rate     Eq. (mix), Sec. 2: for decay time t and phase-space point e,
 *            dGamma/(e^{-Gamma t} N) = (|A|^2+|Abar|^2) cosh(y Gamma t)
 *              + (|A|^2-|Abar|^2) cos(x Gamma t) - 2 Re(A Abar*) sinh(y Gamma t)
 *              - 2 Im(A Abar*) sin(x Gamma t),
 *            A (direct decay) and Abar (decay after D0 -> D0bar mixing)
 *            being coherent sums sum_i c_i A_i over decay chains (Sec. 3),
 *            each chain built from form (barrier) factors, a spin factor,
 *            lineshapes and Bose symmetrisation of the two identical pi-.
 *   norm     Sec. 3.1: normalisation N computed numerically, as the mean
 *            over a flat phase-space Monte Carlo (MC) sample of the rate
 *            integrated over t in [0, inf) in closed form.
 *   NLL      -sum_{data} ln( e^{-Gamma t} B(e) / N ).
 *
 * Units: GeV, ps.  Final-state order: p0 = K+, p1 = pi-, p2 = pi+, p3 = pi-.
 *
 * Parameter vector (length tdmix_num_params):
 *   [Re c_i, Im c_i] for every chain i in model order,
 *   [m0_r, Gamma0_r] for every resonance r in model order,
 *   x, y.
 * Fixed parameters (see tdmix_set_floating) keep their place; their
 * gradient entries are 0.
 *
 * Pointers: arguments documented as "host or device" may point to host
 * memory (the call then synchronises with its stream and returns with the
 * results written) or to device memory (the call is enqueued on the
 * context's stream and returns immediately).  The kind is detected with
 * cudaPointerGetAttributes.  Inputs are copied; outputs are written to the
 * caller's buffers; the context owns all of its device memory.  No C++
 * exception crosses this interface.  One context must not be used from two
 * threads at the same time.
 *
 * Every function returning int returns a tdmix_status; on failure
 * tdmix_last_error describes the cause.
 */
#ifndef TDMIX_H
#define TDMIX_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct tdmix_ctx tdmix_ctx;

typedef enum {
  TDMIX_OK = 0,
  TDMIX_ERR_ARG = -1,       /* invalid argument or model description */
  TDMIX_ERR_NOMEM = -2,     /* device or host allocation failed */
  TDMIX_ERR_CUDA = -3,      /* a CUDA call failed */
  TDMIX_ERR_STATE = -4,     /* no events loaded / wrong call order */
  TDMIX_ERR_NONFINITE = -5, /* non-finite parameter, or a rate <= 0 / not finite */
  TDMIX_ERR_DOMAIN = -6,    /* |y| >= 1, mass or width <= 0, pole below threshold */
  TDMIX_ERR_TIMEOUT = -7,   /* a bounded wait gave up */
  TDMIX_ERR_UNSUPPORTED = -8 /* operation not available for this context (see tdmix_create) */
} tdmix_status;

typedef enum {
  TDMIX_FP64 = 0, /* every per-event quantity in float64 */
  TDMIX_FP32 = 1, /* lineshapes, spin factors and coherent sums in float32;
                     mixing terms, log-likelihood sum and normalisation
                     accumulation in float64 */
  TDMIX_GENERIC = 0x100 /* flag, OR-ed into the precision: evaluate with the
                     runtime-table kernels even where the model's structure
                     has a compiled specialisation (comparisons, tests) */
} tdmix_precision;

/* Which kernels a context evaluates with (tdmix_kernel_path). */
typedef enum {
  TDMIX_PATH_FP64 = 0,   /* structure-specialised kernels, float64 */
  TDMIX_PATH_FP32 = 1,   /* structure-specialised kernels, precision path */
  TDMIX_PATH_GENERIC = 2 /* runtime-table kernels, float64 */
} tdmix_kernel_path_kind;

/* One event sample in structure-of-arrays form.
 *   n          number of events (>= 1)
 *   p[a][c]    n doubles: component c (0:E, 1:px, 2:py, 3:pz) of final-state
 *              particle a, GeV; 16 planes
 *   t          n decay times in ps (data); NULL for phase-space MC
 *   w          n MC event weights; NULL means weight 1 (ignored for data)
 *   on_device  0: all pointers are host memory; 1: all are device memory */
typedef struct {
  int64_t n;
  const double* p[4][4];
  const double* t;
  const double* w;
  int on_device;
} tdmix_events;

/* Creates a context for an amplitude model (Sec. 3: resonances and decay
 * chains assigned to A_f or Abar_f, JSON text; see the shipped model files
 * for the schema) on the current CUDA device.  Recurring building blocks are
 * shared (Sec. 3: recurring form factors, spin factors and lineshapes are
 * linked to one instance).  *out receives the context; TDMIX_ERR_ARG for an
 * invalid model or precision.
 * The kernels are specialised at build time on the structures of the
 * shipped model files (which lineshapes enter which term of which
 * component).  A model of any other structure - the user composes chains,
 * amplitudes and the time-dependent model (Sec. 3) - is evaluated by the
 * runtime-table kernels instead: the same likelihood and gradient, in
 * float64 whatever precision was asked for (so within the tolerances of
 * both paths), several times slower, with every evaluation a full one (no
 * component cache) and without the serving loop (tdmix_server_create
 * returns TDMIX_ERR_UNSUPPORTED) or the device generator (tdmix_generate
 * returns TDMIX_ERR_UNSUPPORTED).  tdmix_kernel_path tells which kernels a
 * context uses; precision | TDMIX_GENERIC selects the runtime-table kernels
 * for any model.
 * A model file may give "time_resolution": sigma (ps), a Gaussian
 * decay-time resolution (an extension; the paper's study has none, Sec. 4).
 * The rate of Eq. (mix) is then folded with it in the measured time t
 * (which may be negative): R(t) = int_0^inf e^{-Gamma t'} B(t') G(t - t';
 * sigma) dt', in closed form through the Faddeeva function; N is unchanged;
 * the NLL is -sum ln(R/N).  Such a model always runs on the runtime-table
 * kernels; |x| Gamma sigma / sqrt 2 must not exceed 0.25 (TDMIX_ERR_DOMAIN);
 * tdmix_generate smears the accepted true times by the resolution.
 * A model file may also give "background": {"fraction": f, "tau": tau_b}
 * (an extension; the paper's study has none, Sec. 4): each data event's
 * density is then (1 - f) R / N + f B, B flat in the normalised phase space
 * (the MC mean has volume 1) and e^{-t/tau_b}/tau_b in the decay time
 * (folded with the resolution if there is one), and the NLL is -sum ln of
 * it.  Also runtime-table kernels only (three passes: MC, N, data);
 * tdmix_event_rates still returns the signal rates R and N. */
int tdmix_create(const char* model_json, int precision, tdmix_ctx** out);

/* The kernels the context evaluates with (tdmix_kernel_path_kind), or a
 * negative status. */
int tdmix_kernel_path(const tdmix_ctx* ctx);

/* Uses the given cudaStream_t (NULL: the legacy default stream) for all
 * later work of the context.  Work already enqueued on the previous stream
 * is waited for first (the context's buffers are then reused on the new
 * one). */
int tdmix_set_stream(tdmix_ctx* ctx, void* cuda_stream);

/* Length of the parameter vector, or a negative status. */
int tdmix_num_params(const tdmix_ctx* ctx);

/* Number of distinct per-event components a_j after sharing (the U of
 * tdmix_norm_matrix), or a negative status. */
int tdmix_num_components(const tdmix_ctx* ctx);

/* Component index of chain `chain` (model order), or a negative status. */
int tdmix_chain_component(const tdmix_ctx* ctx, int chain);

/* Writes the model file's parameter values (host array, num_params). */
int tdmix_default_params(const tdmix_ctx* ctx, double* out);

/* Floating mask (host array of num_params ints, nonzero = floating).  The
 * initial mask comes from the model file. */
int tdmix_set_floating(tdmix_ctx* ctx, const int* mask);

/* Loads the data sample (with decay times) and the phase-space MC sample
 * used for the normalisation (Sec. 3.1), replacing earlier ones.  Copies the
 * events and precomputes, once, every parameter-independent per-event
 * quantity: invariant masses, width factors and spin x barrier factors.
 * Either pointer may be NULL to keep the sample loaded before. */
int tdmix_load_events(tdmix_ctx* ctx, const tdmix_events* data, const tdmix_events* mc);

/* NLL at `params` (host or device, num_params doubles) into *nll_out (host
 * or device) and, if grad_out is not NULL, its gradient (num_params doubles,
 * host or device).  With host params, a call in which no mass or width moved
 * since the previous call (and none floats, or no gradient is asked for)
 * reuses the per-event component cache and the stored MC normalisation
 * matrix; otherwise every step is recomputed.  Host outputs: returns
 * TDMIX_ERR_NONFINITE / TDMIX_ERR_DOMAIN for invalid parameters or a rate
 * <= 0.  Device outputs: such failures are reported as NaN values.
 * One kernel launch does the whole evaluation: host params travel in its
 * arguments, device params are read by it when the stream reaches it; it
 * writes device outputs itself and host outputs through mapped pinned
 * memory, so no separate copy is enqueued. */
int tdmix_nll(tdmix_ctx* ctx, const double* params, double* nll_out, double* grad_out);

/* NLL (and, if grad_out is not NULL, gradient) at n_points parameter
 * vectors, the same computation as tdmix_nll at each: params is a device
 * array [n_points][num_params], nll_out a device array [n_points], grad_out
 * NULL or a device array [n_points][num_params]; all three must be ready
 * when the stream reaches the call (stream-ordered, returns without
 * synchronising).  Every evaluation is a full one (lineshapes, components,
 * MC normalisation, data pass, adjoint).  Consecutive evaluations overlap on
 * the device (programmatic dependent launch): each may start while the one
 * before it finishes, and waits for it before writing anything that is read
 * later (component cache, partial sums, results).  For a minimiser's line
 * search or Hessian columns, a parameter scan, or many fits of one sample.
 * Invalid parameters and rates <= 0 give NaN values, as for device outputs
 * of tdmix_nll.  TDMIX_ERR_ARG for host pointers or n_points < 1. */
int tdmix_nll_batch(tdmix_ctx* ctx, const double* params, int64_t n_points, double* nll_out, double* grad_out);

/* Per-event rate e^{-Gamma t} B(e) of Eq. (mix) for every data event
 * (rates_out: host or device, n_data doubles) and, if norm_out is not NULL,
 * the normalisation N (one double, same memory kind as rates_out).  Always
 * a full evaluation (no component cache), so on the fp32 path every rate
 * is within 1e-5 relative of its double-precision value (see
 * tdmix_recomputed_events). */
int tdmix_event_rates(tdmix_ctx* ctx, const double* params, double* rates_out, double* norm_out);

/* Normalisation matrix I_jk = sum_e w_e a_j(e)^* a_k(e) / sum_e w_e of the
 * components over the MC sample (Sec. 3.1), from the last evaluation that
 * recomputed it; I_out (host) receives U*U complex numbers as interleaved
 * (re, im) pairs, row-major in (j, k). */
int tdmix_norm_matrix(tdmix_ctx* ctx, double* I_out);

/* Pseudo-events of the context's model on the GPU (Sec. 3.1: flat
 * phase-space points and time-dependent pseudo-events by accept/reject).
 * Candidates are flat four-body phase-space points (GENBOD, F. James, CERN
 * 68-15) with decay times t ~ Exp((1 - |y|) Gamma); without TDMIX_GEN_FLAT
 * each is kept with probability R e^{(1-|y|) Gamma t} / env, R = e^{-Gamma t} B
 * the rate of Eq. (mix) at `params` (double precision, whatever the
 * context's precision), env 1.5 times the largest weight of a pilot batch
 * (raised and the sample redrawn, at most four times, if a later weight
 * exceeds it); with TDMIX_GEN_FLAT every phase-space point is kept and t
 * is 0.  Candidates are first weighed in single precision with an error
 * band (1e-3 of the weight plus 1e-4 of its cancellation-free scale), and
 * only those whose decision falls inside the band are weighed in double
 * precision: the decisions of the double-precision rate at a fraction of
 * its cost; TDMIX_GEN_FP64_ONLY weighs every candidate in double precision
 * (the same sample, slower).  Random numbers: Philox4x32-10 (Salmon et al.,
 * SC'11) with key `seed`, counter (candidate index, stream, draw), so the
 * sample depends only on (seed, stream, params, n) and is written in
 * candidate order.
 *   params  host, num_params doubles (ignored with TDMIX_GEN_FLAT)
 *   flags   TDMIX_GEN_FLAT, TDMIX_GEN_FP64_ONLY (bitwise or)
 *   p_out   device, 16 planes of n doubles: component c (E, px, py, pz) of
 *           final-state particle a at p_out[(4a + c) n + i] (the layout of
 *           tdmix_events with on_device = 1)
 *   t_out   device, n decay times (ps), or NULL
 *   info    host, 4 doubles or NULL: envelope, candidates drawn, accepted
 *           fraction, envelope raises; a positive info[0] on entry is used
 *           as the envelope instead of a pilot (pass the envelope of an
 *           earlier call at the same parameters: samples then depend on it)
 * Synchronises with the context's stream; allocates temporary device
 * buffers (stream-ordered).  TDMIX_ERR_NONFINITE if the pilot finds no
 * positive finite rate or the envelope keeps being exceeded. */
enum { TDMIX_GEN_FLAT = 1, TDMIX_GEN_FP64_ONLY = 2 };
int tdmix_generate(tdmix_ctx* ctx, const double* params, int64_t n, uint64_t seed, uint32_t stream, int flags,
                   double* p_out, double* t_out, double* info);

/* Philox4x32-10 of the generator for one (counter, key) (self-test entry;
 * the paper has no counterpart): out receives the four 32-bit words. */
int tdmix_test_philox(const uint32_t* counter, const uint32_t* key, uint32_t* out);

/* How the MC normalisation matrix I_jk (Sec. 3.1) is accumulated:
 *   TDMIX_GRAM_AUTO       (default) per-thread register accumulation up to 8
 *                         shared components; beyond that the tensor cores
 *                         (fp32 path) or shared-memory sums (fp64 path);
 *   TDMIX_GRAM_REGISTERS  per-thread register accumulation (up to 8
 *                         components);
 *   TDMIX_GRAM_TENSOR     tcgen05 tensor-core MMAs over each 256-event MC
 *                         tile on exact fixed-point pieces (three bf16
 *                         integer pieces per value, exact integer sums in the
 *                         MMA, double-float accumulation across tiles; fp32
 *                         path only).
 * Returns TDMIX_ERR_UNSUPPORTED for a mode the context's precision or model
 * cannot use, TDMIX_ERR_ARG for an unknown mode.  Results agree between
 * modes within the fp32 path's tolerance (the modes round differently). */
enum { TDMIX_GRAM_AUTO = 0, TDMIX_GRAM_REGISTERS = 1, TDMIX_GRAM_TENSOR = 2 };
int tdmix_set_gram(tdmix_ctx* ctx, int mode);

/* Number of data events the last evaluation recomputed in double-float
 * (fp32 precision path only; 0 on the fp64 path).  The fp32 amplitudes
 * carry rounding errors of a few ulps of the magnitude of their terms (the
 * decay chains and Bose orderings summed coherently in A and Abar, Sec. 3),
 * so an event whose amplitudes nearly cancel has a large relative error in
 * its rate; a full evaluation recomputes every data event whose estimated
 * term magnitude exceeds 16 times |cosh(w) A - sinh(w) Abar| (Eq. (mix) in
 * factorised form) from double-float inputs.  Synchronises with the
 * context's stream. */
int tdmix_recomputed_events(tdmix_ctx* ctx, int64_t* n);

/* Test hook for the bounded waits: while enabled, block 0 of every
 * evaluation kernel does not issue its first event-tile copy, so its wait for
 * that tile gives up after one second and the evaluation reports
 * TDMIX_ERR_TIMEOUT (host outputs; NaN values with device outputs).  The
 * kernel then returns normally and the context stays usable; the component
 * cache and stored normalisation are marked stale.  Nothing faults or hangs:
 * every wait in the kernels is bounded.  Off by default. */
int tdmix_test_withhold_copy(tdmix_ctx* ctx, int enable);

/* Self-test of the device arithmetic the kernels use in place of CUDA's
 * functions (library extension for testing; the paper has no counterpart).
 * Evaluates routine `which` on n host arguments `in` on the current device
 * and writes n results to `out` (host; 4n for the mixing-series codes:
 * cosh v, sinh v, cos v, sin v per argument).  The Eq. (mix) codes take n
 * records of 8 doubles in `in` and write 4 doubles per record.  Returns TDMIX_ERR_ARG for a
 * bad code, n < 1 or a null pointer, TDMIX_ERR_NOMEM / TDMIX_ERR_CUDA on
 * failure of its own allocations, copies or launch. */
enum {
  TDMIX_MATH_LOG_TABLE = 0, /* table-driven natural logarithm (Tang's method), positive normal v */
  TDMIX_MATH_LOG_CUDA = 1,  /* CUDA's log, for comparison */
  TDMIX_MATH_RCP_F64 = 2,   /* 1/v from the hardware approximation and two Newton steps */
  TDMIX_MATH_DIV_F64 = 3,   /* IEEE double division 1.0 / v, for comparison */
  TDMIX_MATH_RCP_F32 = 4,   /* 1/v in single precision: approximation and one Newton step */
  TDMIX_MATH_DIV_F32 = 5,   /* IEEE single division 1.0f / v, for comparison */
  TDMIX_MATH_DF_RCP = 6,    /* 1/v in double-float arithmetic (v split into two floats) */
  TDMIX_MATH_MIX_TIER0 = 7, /* cosh, sinh, cos, sin by the series through z^3 (|v| <= 0.02) */
  TDMIX_MATH_MIX_TIER1 = 8, /* the same through z^5 (|v| <= 0.1) */
  TDMIX_MATH_MIX_TIER2 = 9, /* CUDA's cosh, sinh, cos, sin, for comparison */
  TDMIX_MATH_LOG_DF = 10,   /* ln v by the double-float table method of the fp32 path (v split into two
                               floats; NaN outside its range) */
  TDMIX_MATH_MIX_DF = 11,   /* Eq. (mix) of the fp32 path in double-float arithmetic: per record
                               {Ar, Ai, Br, Bi, t, x, y, Gamma} (8 input doubles; amplitudes rounded to
                               float, t to a double-float pair) out {ln B, e^{-Gamma t} B, ok, 0} */
  TDMIX_MATH_MIX_F64 = 12,  /* the same records through the fp64 path's Eq. (mix), for comparison */
  TDMIX_MATH_RCP_APPROX_F32 = 13, /* 1/v in single precision by the hardware approximation alone (the
                                     lineshapes' reciprocal on the fp32 path) */
  TDMIX_MATH_CODES = 14
};
int tdmix_test_math(int which, int64_t n, const double* in, double* out);

/* Kernel classes timed by tdmix_profile. */
enum {
  TDMIX_PROF_EVAL = 0,       /* one evaluation: per-evaluation constants, data tiles (components or
                                cache, Eq. (mix), log sum, adjoint), MC tiles (components,
                                normalisation matrix, adjoint), fixed-order reduction, N, NLL, gradient */
  TDMIX_PROF_PRECOMPUTE = 1, /* once per event load: invariants, width and spin x barrier factors */
  TDMIX_PROF_CLASSES = 2
};

/* Enables (1) or disables (0) timing of every kernel the context launches:
 * a CUDA event pair is recorded on the context's stream around each launch.
 * Library extension for measurement; not part of the paper's method. */
int tdmix_profile(tdmix_ctx* ctx, int enable);

/* Accumulated device time in ms (ms_out[TDMIX_PROF_CLASSES]) and launch
 * counts (launches_out[TDMIX_PROF_CLASSES]) of the timed kernels since the
 * last reset; synchronises with the recorded events.  reset != 0 clears the
 * totals afterwards. */
int tdmix_profile_read(tdmix_ctx* ctx, double* ms_out, int64_t* launches_out, int reset);

/* ---- Serving ------------------------------------------------------------
 * Many minimisers fitting independent pseudo-experiments (the paper's
 * sensitivity study, Sec. 4, fits toy samples with a fixed model and
 * floating x, y) submit (sample, parameters) requests concurrently.  The
 * server keeps the model's resonance masses and widths fixed, so the MC
 * normalisation sums are computed once and every resident sample keeps its
 * per-event component cache.  Requests go to a device-resident loop: a
 * persistent kernel on all but 16 SMs takes (request, chunk of event
 * tiles) work items from a ring in page-locked, device-mapped memory as the
 * host publishes them, so requests that arrive while others run are served
 * at once, alongside them; the block finishing a request's last chunk
 * writes its result and a completion flag back to mapped memory.  Samples
 * are admitted into device memory by footprint (2U component values + one
 * decay time per event) on a separate stream and thread, concurrently with
 * the loop; when the budget binds, least recently used samples without
 * pending requests are evicted, and a request whose sample cannot be
 * admitted yet waits for memory to free up.  A request's result does not
 * depend on which other requests are in flight (bitwise).  The loop stops
 * itself after 20 ms without work and is relaunched by the next request;
 * every device-side wait is bounded.  All functions are thread-safe. */
typedef struct tdmix_server tdmix_server;

/* hbm_budget_bytes: device memory allowed for resident samples;
 * max_slots: requests in flight at most (1 .. 1024). */
int tdmix_server_create(const char* model_json, int precision, size_t hbm_budget_bytes, int max_slots,
                        tdmix_server** out);
/* The shared phase-space MC sample (host or device memory, see
 * tdmix_events); computes the normalisation sums of the fixed model. */
int tdmix_server_add_mc(tdmix_server* s, const tdmix_events* mc);
/* Registers a data sample (copied to page-locked host memory; admitted to the
 * device on demand, and again after an eviction); *sample_id receives its id. */
int tdmix_server_add_sample(tdmix_server* s, const tdmix_events* data, int* sample_id);
/* Registers a sample that the server generates on the device each time it
 * admits it (tdmix_generate with the model at `params`, n events, seed and
 * stream): pseudo-experiments need no host copy and are regenerated
 * identically after an eviction; *sample_id receives its id.  The
 * generator's envelope is found once per set of generating parameters and
 * reused for the samples that share them. */
int tdmix_server_add_generated_sample(tdmix_server* s, const double* params, int64_t n, uint64_t seed,
                                      uint32_t stream, int* sample_id);
/* Queues an NLL + gradient evaluation of sample_id at params (host,
 * num_params doubles; masses and widths must equal the model's values,
 * else TDMIX_ERR_ARG).  *ticket identifies the request. */
int tdmix_server_submit(tdmix_server* s, int sample_id, const double* params, uint64_t* ticket);
/* Waits up to timeout_s seconds for a request: *nll and, if grad is not
 * NULL, the gradient (host, num_params doubles; masses and widths get 0).
 * TDMIX_ERR_TIMEOUT if it is not done in time (the request stays valid and
 * can be waited for again); the request's own status otherwise. */
int tdmix_server_wait(tdmix_server* s, uint64_t ticket, double* nll, double* grad, double timeout_s);
/* Latency percentiles (submit to completion, microseconds) and throughput
 * (completed requests per second between the first submit and the last
 * completion) since creation or the last reset. */
int tdmix_server_stats(tdmix_server* s, double* p50_us, double* p99_us, double* evals_per_s);
/* Latency populations of tdmix_server_latency. */
enum tdmix_latency_kind {
  TDMIX_LATENCY_ALL = 0,      /* every completed request (as tdmix_server_stats) */
  TDMIX_LATENCY_RESIDENT = 1, /* requests whose sample was resident when submitted */
  TDMIX_LATENCY_ADMITTED = 2  /* requests that waited for their sample's admission
                               * (upload or generation, component cache) */
};
/* Latency percentiles (submit to completion, microseconds) of one
 * population since creation or the last reset, and its size in *count
 * (each output may be NULL).  An empty population gives NaN percentiles
 * and TDMIX_OK; a kind outside tdmix_latency_kind gives TDMIX_ERR_ARG. */
int tdmix_server_latency(tdmix_server* s, int kind, double* p50_us, double* p99_us, int64_t* count);
int tdmix_server_reset_stats(tdmix_server* s);
/* Device memory currently held by resident samples. */
int tdmix_server_resident_bytes(tdmix_server* s, size_t* bytes);
/* State of the device-resident loop: info[0] launches so far, info[1]
 * launches that ended on their own (a bounded wait gave up; their
 * unfinished requests ran again), info[2] requests published, info[3] 1 if
 * the loop is running, info[4] the device status bits of the last such
 * launch (1: a tile copy did not arrive in time, 2: no work arrived within
 * the loop's idle bound), info[5] how long it had run (microseconds);
 * info holds 6 entries. */
int tdmix_server_loop_info(tdmix_server* s, int64_t* info);
const char* tdmix_server_last_error(const tdmix_server* s);
/* Stops the scheduler (pending requests are dropped) and frees everything. */
void tdmix_server_destroy(tdmix_server* s);

/* Tracing (library extension for measurement; the paper has no
 * counterpart).  With tracing on, every block of the evaluation kernel
 * records TDMIX_TRACE_PHASES globaltimer stamps (ns): start, per-evaluation
 * constants ready, MC tiles done, data tiles done, partials written, then
 * in the last block only: column totals formed, NLL written, end (other
 * blocks repeat their "partials written" stamp there).  Unused rows stay 0. */
#define TDMIX_TRACE_PHASES 8
int tdmix_trace(tdmix_ctx* ctx, int enable);
/* Stamps of the last evaluation: stamps[block * TDMIX_TRACE_PHASES + phase]
 * for *n_blocks blocks (host array of at least (number of SMs) *
 * TDMIX_TRACE_PHASES entries); synchronises with the context's stream. */
int tdmix_trace_read(tdmix_ctx* ctx, unsigned long long* stamps, int* n_blocks);

/* Allocation-free evaluation of sum_e ln B(e) over a component cache the
 * caller keeps itself, where for each event
 *   B = 2 |cosh(w) A - sinh(w) Abar|^2,  w = (y + i x) gamma t / 2,
 *   A = sum_j cA_j a_j,  Abar = sum_j cB_j a_j
 * (the decay-time dependence of the rate without its e^{-gamma t} factor).
 * The paper has no counterpart: this serves callers that cannot allocate
 * device memory while they evaluate, such as work being recorded into a CUDA
 * graph, code running under an external memory manager that owns every
 * device allocation, or a latency-bound loop that must not wait on the
 * allocator.  It calls no cudaMalloc/cudaFree and no allocating library
 * routine: its block partial sums live in a file-scope device array of
 * TDMIX_NOALLOC_MAX_BLOCKS * 2 doubles (16 KiB), which every GPU that loads
 * the library holds until the process exits.
 *   U            number of components, 1 .. 16
 *   n, ld        events, and the plane stride (ld >= n) of a_re / a_im
 *   a_re, a_im   device, [U][ld] doubles: real / imaginary part of a_j(e)
 *   t            device, n decay times (ps)
 *   cA, cB       device, 2U doubles each: coefficient of component j in A_f
 *                and in Abar_f as interleaved (re, im)
 *   x, y, gamma  mixing parameters and the D0 width (1/ps)
 *   out          device, 2 doubles: [sum ln B over events with B > 0,
 *                number of events with B <= 0 or not finite]
 *   stream       cudaStream_t the work is enqueued on (asynchronous)
 * Returns TDMIX_ERR_ARG for U outside 1..16, n < 1, ld < n or a null pointer
 * (any n is accepted: blocks loop over events), TDMIX_ERR_DOMAIN for
 * |y| >= 1 or gamma <= 0, TDMIX_ERR_CUDA if a launch fails.
 * The first call on a device looks up the array's device address with that
 * device current; make that first call before any stream capture starts.
 * Every call shares the array and leaves its partial sums there.  Each call
 * writes every entry it later reads, so nothing needs clearing between
 * calls; but two calls that overlap on the same GPU (for example enqueued on
 * two streams with no ordering between them) race on the array, so such
 * calls must be serialised by the caller. */
#define TDMIX_NOALLOC_MAX_BLOCKS 1024
#define TDMIX_NOALLOC_MAX_DEVICES 64
int tdmix_loglik_components_noalloc(int U, int64_t n, const double* a_re, const double* a_im, int64_t ld,
                                    const double* t, const double* cA, const double* cB, double x, double y,
                                    double gamma, double* out, void* stream);

/* Text of the last failure of this context (never NULL). */
const char* tdmix_last_error(const tdmix_ctx* ctx);

/* Releases the context and all of its device memory. */
void tdmix_destroy(tdmix_ctx* ctx);

#ifdef __cplusplus
}
#endif

#endif /* TDMIX_H */
