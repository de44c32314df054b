/*
 * fdtd.h -- C ABI of the GB300 (sm_103a) FDTD solver for the 1+1D delay PDE
 * of waveguide QED: a two-level system at distance a from a mirror, driven by
 * one or two photons (Fang, "FDTD: solving 1+1D delay PDE in parallel",
 * arXiv:1707.05943).
 *
 * What is computed.  psi(x,t), the amplitude of "atom excited + one photon at
 * x", obeys Eq. 1: advection, decay W = i w0 + Gamma/2, the delay term
 * (Gamma/2) psi(x-2a, t-2a), two mirror source terms (lines 2-3) and the
 * incident two-photon term (line 4).  The library marches Eq. 1 on the square
 * lattice dx = dt = delta (Sec. 2), with squares (Eq. 3a-c) for line 1 and
 * bars (Eq. 4) for lines 2-3, in the region x > -a, column by column left to
 * right and row by row upward.  The exact solution psi(x<=-a,t) = C phi(x-t)
 * e(t) (Sec. 2 (b),(c)) is the boundary; e(t) involves the incomplete Gamma
 * function gamma(n,z) (App. C).
 *
 * Grid.  Column m is x = m delta, row n is t = n delta, D = 2a/delta (even;
 * the paper's n_x).  Marched columns are m = -D/2+1 .. -D/2+nx (index
 * j = m + D/2 - 1 in every buffer below), rows n = 0 .. nt-1.  Row 0 is the
 * initial condition psi(x>-a, 0) = 0.  Complex values are interleaved
 * (re, im): complex128 for FDTD_F64 and FDTD_F64_DW, complex64 for
 * FDTD_F32_COMP.
 *
 * Memory.  The library never allocates device memory.  fdtd_plan reports the
 * workspace size; the caller allocates it (any allocator) and lends it with
 * fdtd_bind_workspace for the plan's lifetime.  The workspace holds a ring of
 * D+2 rows (the delay term reaches row n-D-1), the boundary tables, the
 * per-row norms and the optional snapshots.  The library never frees caller
 * memory.  Host-side plan structs are allocated with malloc and released by
 * fdtd_destroy.
 *
 * Streams and errors.  Every call returns an fdtd_status; nothing throws or
 * exits.  Work is queued on the plan's stream; fdtd_readout synchronises it.
 * Device-side failures (a bounded wait that gave up, a boundary series that
 * did not converge) latch a status word in the workspace that the next
 * fdtd_readout returns.  Plans are not thread-safe; use one plan per stream.
 * Call order: fdtd_plan -> fdtd_bind_workspace -> fdtd_set_boundary ->
 * fdtd_march* -> fdtd_readout*; out-of-order calls return FDTD_ERR_STATE.
 */
#ifndef FDTD_H_
#define FDTD_H_

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct fdtd_plan_s* fdtd_plan_t;

typedef enum {
  FDTD_OK = 0,
  FDTD_ERR_INVALID_ARG = 1,   /* a parameter is out of range (see fdtd_last_error) */
  FDTD_ERR_UNSUPPORTED = 2,   /* valid request this build does not implement       */
  FDTD_ERR_WORKSPACE = 3,     /* workspace missing, too small or misaligned        */
  FDTD_ERR_CUDA = 4,          /* a CUDA runtime call failed                        */
  FDTD_ERR_TIMEOUT = 5,       /* a device-side bounded wait gave up                */
  FDTD_ERR_BOUNDS = 6,        /* reserved: no call of this build returns it (every */
                              /* index a kernel uses is checked on the host first)  */
  FDTD_ERR_NOT_CONVERGED = 7, /* a boundary series or quadrature did not converge  */
  FDTD_ERR_STATE = 8          /* call out of order                                 */
} fdtd_status;

typedef enum {
  FDTD_F64 = 0,       /* complex128 march                                          */
  FDTD_F32_COMP = 1,  /* complex64 march with compensated increments; the boundary */
                      /* tables and the norm reduction stay FP64                   */
  FDTD_F64_DW = 2     /* the FP64 march's results (same tolerance against the FP64 */
                      /* oracle) computed in double-float arithmetic: each value a */
                      /* pair of FP32 numbers (48 significant bits) on the FP32    */
                      /* pipes; readouts are complex128, as for FDTD_F64           */
} fdtd_precision;

typedef enum {
  FDTD_IC_PLANE_WAVE = 1,       /* Sec. 2 (a): two-photon plane wave e^{ik(x1+x2)},  */
                                /* amplitude A = 1 (not normalisable; alpha unused) */
  FDTD_IC_STIM_EMISSION = 2,    /* Sec. 2 (b): atom excited, one exponential photon  */
  FDTD_IC_TWO_PHOTON_EXP = 3,   /* Sec. 2 (c): two identical exponential photons     */
  FDTD_IC_TWO_PHOTON_GAUSS = 4, /* two identical Gaussian photons (same structure as  */
                                /* Sec. 2 (c); e(t) by quadrature, no closed form)    */
  FDTD_IC_TWO_PHOTON_PAIR = 5   /* Sec. 2 (c): two exponential photons (k, alpha) and */
                                /* (k2, alpha2), chi(x1,x2,0) = (A/sqrt2)[phi1(x1)    */
                                /* phi2(x2) + phi1(x2) phi2(x1)] with the paper's A;  */
                                /* FDTD_F64 and FDTD_F64_DW plans                     */
} fdtd_init_cond;

/* Parameters of one instance, in the physical units of the paper's figure
 * captions (c = 1).  Table 1 keys: Nx (here the number of marched columns,
 * not the half-width), Ny = nt, nx = D, Delta = delta, k, w0 = omega0, gamma,
 * init_cond, alpha, Tstep = tstep. */
typedef struct {
  uint32_t struct_size;  /* = sizeof(fdtd_params); versions the ABI              */
  int32_t D;             /* 2a/delta: even, 2 <= D <= nx                         */
  int64_t nx;            /* marched columns, >= D                                */
  int64_t nt;            /* rows, >= 1                                           */
  double delta;          /* grid step > 0                                        */
  double gamma;          /* decay rate Gamma > 0                                 */
  double omega0;         /* two-level-system frequency w0                        */
  double k;              /* incident carrier wavenumber                          */
  int32_t init_cond;     /* fdtd_init_cond                                       */
  int32_t precision;     /* fdtd_precision                                       */
  double alpha;          /* exponential width in units of Gamma (> 0; IC 2, 3)   */
  double sigma;          /* Gaussian width (> 0; IC 4)                           */
  double center;         /* Gaussian centre x_c (IC 4); the pulse is cut at x=-a */
  int32_t tstep;         /* keep every (tstep+1)-th row as a snapshot; -1: none  */
  int32_t rows_per_launch; /* rows marched per kernel launch; 0 = default        */
  int32_t cluster_ctas;  /* FDTD_F32_COMP: most band streams of one instance,    */
                         /* 1..64 (0 = 32): an instance marches in bands of 256  */
                         /* rows, g streams of them in flight at once            */
  int32_t mid_weight;    /* FDTD_F64, FDTD_F64_DW: cost of a column of            */
                         /* -a < x <= 3a in bulk columns in the column split.     */
                         /* FDTD_F32_COMP: stream share s: instance i gets        */
                         /* g = ceil(nx_i nt_i / (sum nx nt / (CTAs s/8))) band   */
                         /* streams, capped by cluster_ctas and its bands.        */
                         /* 1..4096; 0 = 16                                        */
  double k2;             /* FDTD_IC_TWO_PHOTON_PAIR: carrier of the second photon */
  double alpha2;         /* FDTD_IC_TWO_PHOTON_PAIR: its width (> 0)             */
  int64_t max_probes;    /* FDTD_F64 / FDTD_F64_DW: capacity of fdtd_set_probes;  */
                         /* 0 = none                                              */
  int64_t spin_cycles;   /* bound of the march's waits on other CTAs, in SM clock */
                         /* cycles; 0 = 4e9 (~2 s).  A wait that runs out latches */
                         /* FDTD_ERR_TIMEOUT and the march stops (the next        */
                         /* fdtd_readout returns it).  A small value is for tests */
                         /* of that path.                                          */
} fdtd_params;

/* fdtd_set_boundary sources */
enum {
  FDTD_BOUNDARY_ANALYTIC = 0, /* e(t) by the library's gamma(n,z) / quadrature kernel */
  FDTD_BOUNDARY_TABLE = 1,    /* e(r delta), r = 0..nt-1, complex128, given on device */
  FDTD_BOUNDARY_RESTORE = 2   /* analytic boundary, then resume from a checkpoint     */
                              /* (FDTD_READ_STATE of a plan with the same parameters;*/
                              /* any memory, n = its size in bytes)                  */
};

/* fdtd_readout kinds */
enum {
  FDTD_READ_ROW = 0,       /* last marched row: nx complex (precision's type)       */
  FDTD_READ_NORMS = 1,     /* N(n) for n = 0..rows_done-1: FP64                     */
  FDTD_READ_SNAPSHOTS = 2, /* rows 0, tstep+1, 2(tstep+1), ... marched so far       */
  FDTD_READ_ETABLE = 3,    /* e(r delta), r = 0..nt-1: complex128 (PAIR: the first  */
                           /* photon's e0)                                          */
  FDTD_READ_ROWS_DONE = 4, /* int64: rows available (row 0 counts)                  */
  FDTD_READ_STATE = 6,     /* checkpoint: the rows the march still reads (the last  */
                           /* min(rows, D+2), in the plan's storage format), the    */
                           /* compensation remainders (FDTD_F32_COMP), the norms    */
                           /* so far, behind a header of the parameters; a batched  */
                           /* plan gives one such record per instance (by           */
                           /* fdtd_readout_instance).  Snapshots are not included.  */
  FDTD_READ_PROBES = 7,    /* psi at the points of fdtd_set_probes, complex128, in  */
                           /* the order given (0 where the march has not yet been)  */
  FDTD_READ_CHI = 8,       /* chi at the points of fdtd_set_chi_points, complex128  */
  FDTD_READ_MEASURES = 5   /* App. D, per snapshot row n marched so far: 4 doubles  */
                           /* (Re mu, Im mu, lambda, det M = |mu|^2 lambda); needs   */
                           /* FDTD_IC_STIM_EMISSION, tstep >= 0, FDTD_F64/F64_DW.    */
                           /* mu(t) = int phi* psi dx with phi the one-excitation    */
                           /* photon (free packet minus the emission of the atom and */
                           /* its mirror image), lambda(t) = int |psi|^2 dx - |e0|^2; */
                           /* x <= -a exact, x > -a by the trapezoid rule            */
};

/*
 * fdtd_plan -- validate parameters and size the workspace.
 *   p            : array of n_instances parameter sets (host memory, read only;
 *                  copied).  FDTD_F64 plans hold one instance.  FDTD_F32_COMP
 *                  plans hold 1 or more independent instances (each with its own
 *                  nx, nt, D, physics and tstep; rows_per_launch, cluster_ctas
 *                  and mid_weight are taken from p[0]); fdtd_march then advances every instance by n_rows in
 *                  one persistent cooperative launch: an instance is marched in
 *                  bands of 256 rows, up to cluster_ctas band streams at once.
 *   cuda_stream  : cudaStream_t the plan queues its work on (NULL = default).
 *   workspace_bytes (out): device bytes the caller must lend (256-byte aligned).
 *   out (out)    : new plan handle, released by fdtd_destroy.
 * Derivation (Sec. 2, Eq. 3a-c, App. A): a = D delta / 2, W = i w0 + Gamma/2,
 * A = 1/delta + W/4; the update coefficients are (1/delta - W/4)/A, -(W/4)/A,
 * (Gamma/8)/A and 1/A.  Errors: FDTD_ERR_INVALID_ARG (D odd, D > nx, delta <= 0,
 * ...), FDTD_ERR_UNSUPPORTED, FDTD_ERR_CUDA.
 */
fdtd_status fdtd_plan(const fdtd_params* p, int32_t n_instances, void* cuda_stream, size_t* workspace_bytes,
                      fdtd_plan_t* out);

/* fdtd_bind_workspace -- lend `bytes` of device memory at `device_ptr`
 * (256-byte aligned, >= the size fdtd_plan reported) for the plan's lifetime.
 * Errors: FDTD_ERR_WORKSPACE, FDTD_ERR_STATE. */
fdtd_status fdtd_bind_workspace(fdtd_plan_t plan, void* device_ptr, size_t bytes);

/*
 * fdtd_set_boundary -- build the boundary and reset the march to row 0.
 * Computes e(t) on the rows (Sec. 2 (b) e1 series; Sec. 2 (c) e0 series with
 * gamma(n+1,-ip(t-2na)) from App. C; quadrature for Gaussian photons), the
 * wavepacket table phi(-a - j delta), the per-row source scalars, and zeroes
 * the ring.  source = FDTD_BOUNDARY_TABLE takes e(r delta) from device_table
 * (n = nt complex128 values, device memory, read during the call's kernels)
 * instead of computing it.  Asynchronous.  source = FDTD_BOUNDARY_RESTORE
 * builds the analytic boundary and then loads a checkpoint (device_table: the
 * FDTD_READ_STATE bytes of a plan with the same parameters, host or device
 * memory, n = their size; for a batched plan the records of every instance in
 * order); the march resumes at the checkpoint's row, and continuing it gives
 * bitwise the results of the uninterrupted march.  This source synchronises
 * the stream.  Errors: FDTD_ERR_STATE (no workspace), FDTD_ERR_INVALID_ARG
 * (including a checkpoint of other parameters or cut short), FDTD_ERR_CUDA.
 */
fdtd_status fdtd_set_boundary(fdtd_plan_t plan, int32_t source, const void* device_table, int64_t n);

/*
 * fdtd_march -- march n_rows more rows (clamped to nt), asynchronously on the
 * plan's stream.  Each row n solves Eq. 1's discretisation at every marched
 * column; the delay term reads rows n-D and n-D-1 from the ring.  Errors:
 * FDTD_ERR_STATE (no boundary), FDTD_ERR_INVALID_ARG (n_rows < 0),
 * FDTD_ERR_CUDA.
 */
fdtd_status fdtd_march(fdtd_plan_t plan, int64_t n_rows);

/*
 * fdtd_march_graph -- fdtd_march for FDTD_F32_COMP plans through a CUDA graph.
 * The first call for a given (clamped) n_rows records the launch sequence of
 * the march (descriptor advance, queue reset and one persistent launch per
 * rows_per_launch rows) on an internal stream and instantiates it; later calls
 * with the same n_rows replay it.  The replay is ordered after the work already
 * queued on the plan's stream, and later work on that stream after it (events).
 * The graph, the internal stream and its events are driver resources held by
 * the plan until fdtd_destroy.  Results are bitwise those of fdtd_march.
 * Errors: as fdtd_march, FDTD_ERR_UNSUPPORTED for FDTD_F64 plans.
 */
fdtd_status fdtd_march_graph(fdtd_plan_t plan, int64_t n_rows);

/*
 * fdtd_readout -- synchronise the plan's stream and copy `kind` into dst.
 *   dst       : caller-owned host or device memory (cudaMemcpyDefault).
 *   dst_bytes : capacity of dst; FDTD_ERR_INVALID_ARG if too small.
 * Returns a latched device error (FDTD_ERR_TIMEOUT, FDTD_ERR_NOT_CONVERGED)
 * first.
 * Norms: N(n) = delta * trapezoid of |psi(x, n delta)|^2 over x = -a (exact
 * boundary value) .. the last marched column, accumulated in FP64 (App. D).
 */
fdtd_status fdtd_readout(fdtd_plan_t plan, int32_t kind, void* dst, int64_t dst_bytes);

/*
 * fdtd_set_probes -- points at which the march records psi as it completes
 * their rows (Table 1's save_chi output and Eq. 2 need psi at chosen retarded
 * points, not whole rows).  points: host memory, count pairs (n, j) of row
 * n in [0, nt) and column index j in [0, nx) (x = (j + 1 - D/2) delta), in any
 * order, repeats allowed; count <= max_probes of the plan.  Call after
 * fdtd_set_boundary (which clears the probes); points on rows marched before
 * the call read 0.  FDTD_READ_PROBES returns the values in the order given.
 * FDTD_F64 and FDTD_F64_DW plans.  Errors: FDTD_ERR_STATE (no boundary),
 * FDTD_ERR_INVALID_ARG (a point outside the box, count > max_probes),
 * FDTD_ERR_UNSUPPORTED (FDTD_F32_COMP plans), FDTD_ERR_CUDA.
 */
fdtd_status fdtd_set_probes(fdtd_plan_t plan, const int64_t* points, int64_t count);

/*
 * fdtd_set_chi_points -- the two-photon wavefunction chi(x1, x2, t) by Eq. 2
 * (the formal solution in terms of psi; Table 1's save_chi writes
 * chi(a+delta, a+delta+tau, t)) at grid points: pts, host memory, count
 * triples (i1, i2, n) for x1 = i1 delta, x2 = i2 delta, t = n delta.
 *   chi = chi(x1-t, x2-t, 0) - (sqrt(Gamma)/2) [ T(x1,x2) + T(x2,x1) ],
 *   T(y1,y2) = psi(y1-y2-a, t-y2-a) theta(y2+a) theta(t-y2-a)
 *            - psi(y1-y2+a, t-y2+a) theta(y2-a) theta(t-y2+a),   theta(0) = 1/2;
 * psi at x <= -a is the exact boundary, psi at marched points is recorded by
 * probes that this call registers (replacing those of fdtd_set_probes; at most
 * 4 per point, count <= max_probes / 4).  Call after fdtd_set_boundary and
 * before the rows the points need are marched; FDTD_READ_CHI evaluates chi
 * from the recorded values.  FDTD_F64 / FDTD_F64_DW plans.  Errors:
 * FDTD_ERR_INVALID_ARG (a term right of the box, beyond nt or the wavepacket
 * table, count too large), FDTD_ERR_STATE (no boundary, or a needed row
 * already marched), FDTD_ERR_UNSUPPORTED (batched plans), FDTD_ERR_CUDA.
 */
fdtd_status fdtd_set_chi_points(fdtd_plan_t plan, const int64_t* pts, int64_t count);

/* Size in bytes that fdtd_readout(kind) writes at the current state. */
int64_t fdtd_readout_bytes(fdtd_plan_t plan, int32_t kind);

/*
 * fdtd_readout_instance -- fdtd_readout for instance `instance` of a plan made
 * with n_instances > 1 (instance 0 is what fdtd_readout returns).  For a
 * FDTD_BOUNDARY_TABLE source of a batched plan, device_table holds the
 * instances' tables one after another (sum of nt complex128 values).
 * Errors: FDTD_ERR_INVALID_ARG (instance out of range), as fdtd_readout.
 */
fdtd_status fdtd_readout_instance(fdtd_plan_t plan, int32_t instance, int32_t kind, void* dst, int64_t dst_bytes);

/* Size in bytes that fdtd_readout_instance(instance, kind) writes; -1 if invalid. */
int64_t fdtd_readout_instance_bytes(fdtd_plan_t plan, int32_t instance, int32_t kind);

/* fdtd_destroy -- release the host-side plan (not the workspace). NULL is a no-op. */
void fdtd_destroy(fdtd_plan_t plan);

/* Static description of a status code. */
const char* fdtd_status_string(fdtd_status s);

/* Last error message recorded on the plan (empty string if none). */
const char* fdtd_last_error(fdtd_plan_t plan);

/*
 * fdtd_gamma_star -- the App. C routine on its own: for i < count,
 *   out[i] = Gamma(n[i]) * gamma*(n[i], z[i]) = int_0^1 s^(n-1) e^(-z s) ds,
 * so gamma(n,z) = z^n out and P(n,z) = z^n out / (n-1)!.  n[i] >= 1 (int32),
 * z and out are interleaved complex128.  All three pointers are device memory;
 * the kernel runs on cuda_stream and the call returns without synchronising.
 * Errors: FDTD_ERR_INVALID_ARG (count < 0 or a NULL pointer), FDTD_ERR_CUDA.
 */
fdtd_status fdtd_gamma_star(const int32_t* n, const double* z, double* out, int64_t count, void* cuda_stream);

/*
 * fdtd_march_noalloc -- the whole FP64 march of one instance (boundary, every
 * row, readout) for callers that cannot allocate device memory.  The paper
 * has no counterpart; this is a deployment convenience.
 *
 * Who cannot allocate: a host framework that owns all device memory through
 * its own pool and forbids other allocations, or a plugin inside such a
 * process that may use only the buffers the host hands it.  They can pass
 * inputs and outputs, but cannot lend the march its scratch
 * (fdtd_bind_workspace).
 *
 * Scratch: a 64 MiB array built into the library (fdtd_noalloc_max_bytes()),
 * placed on every GPU that loads the library and held there until the process
 * exits.  An instance whose workspace (as fdtd_plan reports it, without
 * snapshots) exceeds that size is rejected with FDTD_ERR_WORKSPACE before any
 * device work.  Every call on a device shares the array: calls whose work
 * overlaps on the GPU (other streams, other host threads) race and corrupt
 * each other; serialise them.  Each call zeroes the ring, norms and barrier
 * words it uses, so a call does not see the previous call's contents.
 *
 * Set-up: the first call on each device looks up the array's device address
 * (cudaGetSymbolAddress, with that device current).  No call allocates device
 * memory, and none calls cudaMalloc, cudaFree or an allocating library
 * routine.  The call is blocking: it synchronises cuda_stream before it
 * returns, on success and on every error after work was queued, so no work
 * of a failed call is left running on the shared array.
 *
 *   p          : parameters, as for fdtd_plan (precision FDTD_F64; tstep is
 *                ignored: no snapshots are kept).
 *   cuda_stream: cudaStream_t for all work.
 *   row_out    : device memory, nx complex128: psi on the last row nt-1.
 *   norms_out  : device memory, nt doubles: N(n) as FDTD_READ_NORMS defines it.
 * Errors: as fdtd_plan / fdtd_set_boundary / fdtd_march / fdtd_readout, plus
 * FDTD_ERR_WORKSPACE (instance larger than the built-in scratch).
 */
fdtd_status fdtd_march_noalloc(const fdtd_params* p, void* cuda_stream, void* row_out, double* norms_out);

/* Size in bytes of the built-in scratch of fdtd_march_noalloc. */
size_t fdtd_noalloc_max_bytes(void);

/*
 * fdtd_geometric_measure -- the geometric non-Markovianity measure of App. D,
 *   N_geo = integral of d|det M_t|/dt over the times where it is positive,
 * from samples det_m[0..n) of det M_t (FDTD_READ_MEASURES, 4th column), as the
 * sum of the increases of |det M| between consecutive samples.  Host memory,
 * host code.  Errors: FDTD_ERR_INVALID_ARG (NULL, n < 0).
 */
fdtd_status fdtd_geometric_measure(const double* det_m, int64_t n, double* out);

/*
 * fdtd_alu_probe -- measured arithmetic peak of the current GPU, the
 * denominator of the marches' arithmetic roofline (the paper has no
 * counterpart; its march is memory-bound on CPUs).
 *   kind       : 0 FP64 FMA, 1 FP32 FMA, 2 packed FP32 pairs (fma.rn.f32x2).
 *   cuda_stream: stream the probe kernels run on (one untimed, one timed
 *                launch of independent FMA chains on every SM).
 *   flops_per_s (out): 2 flops per FMA (4 per packed FMA) over the timed
 *                launch, measured with CUDA events; the call synchronises.
 * Errors: FDTD_ERR_INVALID_ARG (kind, NULL), FDTD_ERR_CUDA.
 */
fdtd_status fdtd_alu_probe(int32_t kind, void* cuda_stream, double* flops_per_s);

/* ---- surrogate network -----------------------------------------------------
 * The paper has no counterpart: a multilayer perceptron maps a few physical
 * parameters of an instance (for example Gamma a, k0 a, the photon width and
 * centre) to quantities the march produces (the norm N(t) of Sec. 3 on a time
 * grid, a sub-sampled outgoing amplitude), trained on march output.  The march
 * stays the fallback and the judge of the network's error.
 *
 * Network: dims[0] inputs -> GELU(affine) -> ... -> affine -> dims[n_layers]
 * outputs, GELU(z) = z/2 (1 + erf(z/sqrt 2)).  Parameters, one block per layer
 * l = 0..n_layers-1, in this order: W_l [dims[l+1]][dims[l]] row-major, then
 * b_l [dims[l+1]].  All arrays below are device memory owned by the caller,
 * sized fdtd_mlp_param_count elements.  Arithmetic: layer 0 (dims[0] <= 64
 * inputs) in FP32 on the CUDA cores; every other layer on the tensor cores with
 * BF16 weights (params_bf16) and BF16 activations, FP32 accumulation, FP32
 * bias and pre-activations; Adam updates the FP32 masters (params) and then
 * refreshes params_bf16.
 * Shapes: 2 <= n_layers <= 7; dims[1..n_layers] multiples of 64; batch a
 * multiple of 64; params_bf16 16-byte aligned; ws 256-byte aligned.  Calls queue work on cuda_stream and return without
 * synchronising.  Errors: FDTD_ERR_INVALID_ARG (shape rule, NULL pointer,
 * struct_size), FDTD_ERR_CUDA.
 */
typedef struct fdtd_mlp {
  uint32_t struct_size; /* sizeof(fdtd_mlp) */
  int32_t n_layers;     /* affine layers                                  */
  int32_t dims[8];      /* widths: dims[0] inputs .. dims[n_layers] outputs */
  float* params;        /* FP32 master parameters                          */
  void* params_bf16;    /* BF16 copy of params, same layout                */
  float* grads;         /* FP32 gradient of the loss, same layout          */
  float* adam_m;        /* Adam first moment (zero before step 1)          */
  float* adam_v;        /* Adam second moment (zero before step 1)         */
} fdtd_mlp;

/* Number of parameters (floats) of the network. */
fdtd_status fdtd_mlp_param_count(const fdtd_mlp* net, int64_t* count);

/* Device scratch (bytes) that forward / train_step need for `batch` rows. */
fdtd_status fdtd_mlp_workspace_bytes(const fdtd_mlp* net, int32_t batch, size_t* bytes);

/* params_bf16 <- round-to-nearest BF16 of params. */
fdtd_status fdtd_mlp_sync_bf16(const fdtd_mlp* net, void* cuda_stream);

/* y[batch][dims[n_layers]] (FP32) = network(x[batch][dims[0]] (FP32)).
 * ws: device scratch of fdtd_mlp_workspace_bytes, 256-byte aligned. */
fdtd_status fdtd_mlp_forward(const fdtd_mlp* net, const float* x, int32_t batch, float* y, void* ws,
                             void* cuda_stream);

/* One training step on the mean squared error
 *   loss = (1 / (batch * dims[n_layers])) sum (y - target)^2:
 * forward, backward into net->grads (every parameter), and, when lr > 0, one
 * Adam step (beta1 0.9, beta2 0.999, eps 1e-8, bias correction with the 1-based
 * `step`).  *loss (device, FP32) receives the loss of the forward pass.  With
 * lr = 0 the weights stay untouched (gradient only; adam_m / adam_v may be
 * NULL). */
fdtd_status fdtd_mlp_train_step(const fdtd_mlp* net, const float* x, const float* target, int32_t batch, float lr,
                                int32_t step, void* ws, float* loss, void* cuda_stream);

/* The surrogate's GEMM on its own: C[M][N] (FP32, row-major, device) =
 * sum_k A[m lda + k] B[n ldb + k], A and B BF16 device arrays with K
 * contiguous (16-byte aligned, lda and ldb multiples of 8, >= K).  M, N
 * multiples of 64, K a multiple of 32.  Runs on the tensor cores (operands
 * staged by TMA, tcgen05 MMA, FP32 accumulation in tensor memory). */
fdtd_status fdtd_gemm_bf16(const void* A, const void* B, float* C, int32_t M, int32_t N, int32_t K, int32_t lda,
                           int32_t ldb, void* cuda_stream);

/* Synchronise cuda_stream and report (then clear) a GEMM wait that ran out of
 * time on this device since the last call: FDTD_ERR_TIMEOUT, else FDTD_OK.
 * The kernels skip their output after such a timeout instead of hanging. */
fdtd_status fdtd_mlp_status(void* cuda_stream);

#ifdef __cplusplus
}
#endif

#endif /* FDTD_H_ */
