/*
 * gsm.h -- C ABI of the GB300 (sm_103a) library for generalized standard
 * materials (GSM) and the Moulinec-Suquet basic scheme.
 *
 * Method: AutoMat (Bluehdorn, Gauger, Kabel; arXiv 2006.04391).
 *   Sec. 2, Eq. (gsm_sigma), (gsm_internal): a GSM is given by a free energy
 *     psi(eps, z) and a dissipation potential phi (the convex dual of the
 *     paper's force potential Psi); sigma = d psi/d eps.
 *   Sec. 4.1, Eq. (implicit_euler): one implicit Euler step per voxel,
 *     d psi/dz (eps, z) + d phi/dzdot ((z - z_n)/h) = 0, solved by Newton with
 *     first and second derivatives of psi and phi from reverse-mode AD.
 *   Sec. 4.1, Eq. (tangent_formula): consistent tangent by the implicit
 *     function theorem.
 *   Sec. 3 "Material Law Evaluations": the basic scheme calls the law once
 *     per voxel and iteration without tangent; fixed reference stiffness.
 *
 * Conventions for every field array:
 *   - Voigt order (11, 22, 33, 23, 13, 12).  Strain-like arrays (eps, z_n, z,
 *     macroscopic strains E) carry ENGINEERING shears (g_ij = 2 eps_ij);
 *     stress-like arrays (sigma, Sigma) carry tensor shears.  The tangent maps
 *     strain-like to stress-like vectors.
 *   - Structure of arrays: component c of voxel i is at base[c * ld + i].
 *   - Tangent: 21 components, the upper triangle of the symmetric 6x6 matrix
 *     in row-major order (C11, C12, ..., C16, C22, ..., C66), SoA as above.
 *   - All field pointers are DEVICE pointers owned by the caller unless a
 *     function says otherwise.  The library never frees them.
 *   - Calls are asynchronous on the given CUDA stream (NULL = legacy default
 *     stream) unless documented as synchronous.
 *   - Return value: GSM_OK (0) or a negative GSM_E* code; no exception ever
 *     crosses the ABI.  gsm_strerror() gives a static message.
 *
 * Per-voxel status word (int32, optional output of gsm_update):
 *   bits 0-7 line-search iterations, bits 8-15 Newton iterations (including
 *   FP64 corrections), bit 16 converged, bit 17 non-finite input or result,
 *   bit 18 iteration cap reached, bit 19 Newton matrix not positive definite,
 *   bits 20-23 FP64 corrections (GSM_FP32_FP64FIX), bits 24-30 scalar
 *   iterations of the segment model that starts the line search.
 */
#ifndef GSM_GB300_H
#define GSM_GB300_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* ------------------------------------------------------------------ errors */
#define GSM_OK 0
#define GSM_EINVAL (-1)    /* bad argument: kind, parameter, pointer, size */
#define GSM_ENOMEM (-2)    /* device or host allocation failed             */
#define GSM_ECUDA (-3)     /* a CUDA or cuFFT call failed                  */
#define GSM_ENOTCONV (-4)  /* iteration cap reached (see status / result)  */
#define GSM_ENOTSUP (-5)   /* combination not supported                    */

/* ------------------------------------------------------------------- kinds */
#define GSM_PSI_ELASTIC 0        /* psi = 1/2 eps:C:eps, no internal variables      */
#define GSM_PSI_ELASTIC_VP_DEV 1 /* psi = 1/2 (eps-z):C:(eps-z), z deviatoric (5 dof) */
#define GSM_PSI_ELASTIC_VP_KIN 2 /* Eq. michel_suquet_omega: 1/2 (eps-z):C:(eps-z) + 1/3 z:Hv:z
                                    + sigma_Y alpha, z deviatoric (5 dof) and alpha      */
#define GSM_PHI_NONE 0
#define GSM_PHI_NORTON 1         /* phi = sigma0 edot0 n/(n+1) (|zdot|_eq/edot0)^((n+1)/n) */
#define GSM_PHI_MS_FORCE 2       /* Eq. michel_suquet_psi (a FORCE potential Psi(A)):
                                    sigma_d edot0/(n+1) ((|dev A_z|_eq + A_alpha)^+/sigma_d)^(n+1) */

#define GSM_FP64 0               /* every step in FP64                                 */
#define GSM_FP32_FP64FIX 1       /* FP32 Newton, then FP64 correction (FP64 in/out)    */
#define GSM_FP32 2               /* FP32 in, out and arithmetic                        */

typedef struct gsm_material* gsm_handle;

/*
 * gsm_create -- define a material law (Sec. 2: the law is its two potentials).
 *   psi_kind, phi_kind: GSM_PSI_ELASTIC with GSM_PHI_NONE, or
 *                       GSM_PSI_ELASTIC_VP_DEV with GSM_PHI_NORTON, or
 *                       GSM_PSI_ELASTIC_VP_KIN with GSM_PHI_MS_FORCE (the paper's
 *                       Michel-Suquet law, K(alpha) = sigma_Y; integrated by
 *                       gsm_update_ode23 only: its yield function has no smooth
 *                       dissipation form for the implicit-Euler Newton).
 *   params: host array; {E, nu} (n_params = 2) for the elastic law,
 *           {E, nu, sigma0, edot0, n} (n_params = 5) for the Norton law,
 *           {E, nu, sigma_Y, H, edot0, sigma_d, n} (n_params = 7) for the
 *           Michel-Suquet law.  Requires E > 0, -1 < nu < 0.5, sigma0 > 0,
 *           edot0 > 0, n > 0; sigma_Y >= 0, H >= 0, sigma_d > 0, n >= 1.
 *   precision: GSM_FP64, GSM_FP32_FP64FIX or GSM_FP32.
 *   out: receives an opaque handle owned by the library (gsm_destroy).
 * Synchronous, host only.  Errors: GSM_EINVAL, GSM_ENOMEM.
 */
int gsm_create(gsm_handle* out, int psi_kind, int phi_kind, const double* params, int n_params,
               int precision);

/* gsm_destroy -- release a handle (NULL is accepted). */
int gsm_destroy(gsm_handle h);

/*
 * gsm_update -- one implicit-Euler material update of n_vox independent
 * voxels (Sec. 4.1, Eq. implicit_euler; tangent by Eq. tangent_formula).
 *   eps     [6][ld]  strain at t_{n+1}               (in)
 *   z_n     [6][ld]  internal variables at t_n        (in; deviatoric, the
 *                    33 component is recomputed as -z11-z22; ignored and may
 *                    be NULL for the elastic law)
 *   h       step size t_{n+1} - t_n > 0
 *   sigma   [6][ld]  stress at t_{n+1}               (out)
 *   z       [6][ld]  internal variables at t_{n+1}    (out; copy of z_n for
 *                    the elastic law, may be NULL then)
 *   tangent [21][ld] consistent tangent               (out, may be NULL)
 *   status  [ld]     per-voxel status word            (out, may be NULL)
 * Element type: double for GSM_FP64 and GSM_FP32_FP64FIX, float for
 * GSM_FP32.  ld >= n_vox.  n_vox = 0 is a no-op.  Arrays must not overlap.
 * Each array may be device memory or page-locked host memory
 * (cudaHostAlloc / cudaHostRegister): the kernel then reads and writes the
 * host memory directly over the host link (NVLink-C2C on GB300), with no
 * staging copies.  Unregistered host memory is refused with GSM_EINVAL.
 * Asynchronous on `stream` (a cudaStream_t).  Errors: GSM_EINVAL, GSM_ECUDA.
 * A voxel that hits the Newton cap is reported in `status`, not by the
 * return value.
 */
int gsm_update(gsm_handle h, int64_t n_vox, const void* eps, const void* z_n, int64_t ld, double step_h,
               void* sigma, void* z, void* tangent, int32_t* status, void* stream);

/*
 * gsm_update_host -- gsm_update for arrays that live in page-locked host memory,
 * streamed through the device in chunks of `chunk` voxels (0: 2^20): the
 * host->device copies of chunk i+1 and the device->host copies of chunk i-1
 * (two internal streams, the copy engines of both directions of the host link)
 * overlap the update of chunk i (on `stream`).  Same arguments, layouts and
 * results as gsm_update (bit-identical to it on device copies of the arrays);
 * every non-NULL array must be page-locked host memory (cudaHostAlloc /
 * cudaHostRegister), else GSM_EINVAL.  Device staging buffers for three
 * chunks come from the stream-ordered allocator of the current device and go
 * back to it on `stream`.  Asynchronous on `stream`: the results are in host
 * memory once `stream` has passed this call.  Errors: GSM_EINVAL, GSM_ENOMEM,
 * GSM_ENOTSUP, GSM_ECUDA.
 */
int gsm_update_host(gsm_handle h, int64_t n_vox, const void* eps, const void* z_n, int64_t ld, double step_h,
                    void* sigma, void* z, void* tangent, int32_t* status, int64_t chunk, void* stream);

/*
 * gsm_update_ode23 -- material update by adaptive explicit Runge-Kutta
 * integration of the force-potential form ydot = dPsi/dA(-d psi/dy) over the
 * load step (Sec. 4.3: the Bogacki-Shampine 3(2) pair of MATLAB's ode23, step
 * sizes after Hairer-Norsett-Wanner, whole step as the first trial), with the
 * stress-driven error control of Sec. 4.5 and, when tangent != NULL, the
 * tangent ODE of Corollary 1 integrated with the same substeps.
 *   eps_n   [6][ld]  strain at t_n                       (in)
 *   eps     [6][ld]  strain at t_{n+1}                   (in); the strain is
 *                    interpolated linearly in between
 *   z_n     [nz][ld] internal variables at t_n           (in): nz = 6 for the
 *                    Norton law (z, deviatoric), nz = 7 for the Michel-Suquet
 *                    law (z, then the equivalent plastic strain alpha)
 *   h       step size > 0;  rtol > 0, atol >= 0: error tolerances on the
 *           stresses (and tangents); MATLAB's defaults are 1e-3 and 1e-6
 *   max_substeps  cap on accepted + rejected substeps per voxel (>= 1)
 *   sigma [6][ld], z [nz][ld] (out); tangent [36][ld] dsigma/deps_{n+1} as the full
 *           6x6 matrix row-major (not symmetric in general), or NULL
 *   status  [ld] or NULL: bits 0-15 accepted substeps, bits 20-30 rejected
 *           substeps (both saturating), bits 16-19 flags as for gsm_update
 *           (a voxel that reaches max_substeps has bit 18 and keeps the state
 *           of its last accepted substep)
 * Element type double: computed in FP64 whatever the material's precision.
 * The viscoplastic laws only (GSM_ENOTSUP for the elastic law).  Arrays as
 * for gsm_update (device or page-locked host memory).  Asynchronous on
 * `stream`.  Errors: GSM_EINVAL, GSM_ENOTSUP, GSM_ECUDA.
 */
int gsm_update_ode23(gsm_handle h, int64_t n_vox, const void* eps_n, const void* eps, const void* z_n, int64_t ld,
                     double step_h, double rtol, double atol, int max_substeps, void* sigma, void* z, void* tangent,
                     int32_t* status, void* stream);

/* Explicit Runge-Kutta pairs of Sec. 4.3. */
#define GSM_ODE23 0              /* Bogacki-Shampine 3(2) (MATLAB's ode23)              */
#define GSM_ODE12 1              /* explicit Euler (order 1) / Heun (order 2), continued
                                    with Heun's solution; step exponent 1/2            */
#define GSM_ODE23S 2             /* Shampine-Reichelt modified Rosenbrock triple
                                    (MATLAB's ode23s): linearly implicit, for stiff
                                    steps; its tangent uses a hand third derivative
                                    of the force potential (Sec. 4.3)                  */

/*
 * gsm_update_ode -- gsm_update_ode23 with the integrator chosen by `method`
 * (GSM_ODE23, GSM_ODE12 or GSM_ODE23S; anything else: GSM_EINVAL).  Same
 * arguments, layouts, status word and errors; gsm_update_ode23 is method
 * GSM_ODE23.  ode12 evaluates the right-hand side twice per substep and needs
 * about tol^(-1/2) substeps (ode23: tol^(-1/3)); ode23s solves three NY x NY
 * linear systems per substep and is not limited by stiffness.
 */
int gsm_update_ode(gsm_handle h, int method, int64_t n_vox, const void* eps_n, const void* eps, const void* z_n,
                   int64_t ld, double step_h, double rtol, double atol, int max_substeps, void* sigma, void* z,
                   void* tangent, int32_t* status, void* stream);

/* gsm_strerror -- static message for a return code. */
const char* gsm_strerror(int code);

/* gsm_kernel_launches -- number of kernels this library has launched in the
 * calling process (all entry points, all devices); for instrumentation. */
int64_t gsm_kernel_launches(void);

/* gsm_peak_probe -- SIMT FMA-throughput probe, for the rooflines of the
 * material kernels (the paper has no counterpart: it measures no roofline).
 * Launches one kernel on `stream` (asynchronous): blocks_per_sm x (SM count)
 * blocks of 512 threads, each thread running 8 independent dependent chains
 * x <- fma(x, a, b) for `iters` steps in FP64 (precision 0) or FP32 (1).
 * The caller times the launch on `stream`; the FLOP rate is
 * 2 * (*fmas_out) / time.  Allocates nothing; *fmas_out (host) receives the
 * number of FMAs the launch performs.  Errors: GSM_EINVAL (precision not 0
 * or 1, iters outside [1, 2^32], blocks_per_sm outside [1, 64], fmas_out
 * NULL), GSM_ECUDA. */
int gsm_peak_probe(int precision, int64_t iters, int blocks_per_sm, double* fmas_out, void* stream);

/* ================================================ Moulinec-Suquet basic scheme
 *
 * Periodic unit cell discretised by N^3 voxels; voxel (i, j, k) with k the
 * fastest index has linear index (i*N + j)*N + k.  Each voxel carries a phase
 * id (uint8) that selects one of n_phases materials.  Reference medium:
 * isotropic, Lame constants at the midpoints of the phases' elastic ranges
 * (fixed C^ref, Sec. 3).  Load step k: eps <- eps + (E_k - E_{k-1}), then
 * iterate
 *     sigma = law(eps, z_n, h_k)               (material kernel)
 *     sigma^ = FFT(sigma)                      (cuFFT R2C)
 *     e = sqrt(sum_xi |xi.sigma^/N^3|^2) / |<sigma>|_F   (FP64 reduction)
 *     eps^(xi) -= Gamma0(xi) : sigma^(xi), eps^(0) = N^3 E_k   (fused kernel)
 *     eps = IFFT(eps^)                         (cuFFT C2R)
 * until e < tol; then z_n <- z and Sigma_k = <sigma> (FP64).  xi = 2 pi k with
 * k the signed integer frequency; on even grids a mode with the Nyquist index
 * together with any other nonzero index has Gamma0 := 0 and is left out of e.
 */

#define MS_PREC_FP64 0       /* all fields, FFTs and laws in FP64                  */
#define MS_PREC_FP32_BULK 1  /* FP32 fields/FFTs/laws until e < switch_tol or e
                                stalls, then FP64 iterations to tol; residual and
                                mean-stress reductions always in FP64           */

typedef struct ms_problem {
  int N;                      /* grid size per axis, 2 <= N <= 1024            */
  const uint8_t* phase;       /* device [N^3] phase ids < n_phases             */
  int n_phases;               /* 1 .. 16                                       */
  const gsm_handle* laws;     /* host [n_phases] materials; a viscoplastic law
                                 created with GSM_FP32_FP64FIX or GSM_FP32 is
                                 evaluated as FP32 Newton + FP64 correction in
                                 the FP64 iterations, GSM_FP64 in FP64      */
  int precision;              /* MS_PREC_*                                     */
} ms_problem;

typedef struct ms_load {
  int n_steps;                /* number of load steps >= 1                     */
  const double* E;            /* host [n_steps][6] macroscopic strains E_k     */
  const double* h;            /* host [n_steps] step sizes h_k > 0             */
  double tol;                 /* equilibrium tolerance on e                    */
  int max_iter;               /* iteration cap per step (material evaluations) */
  const int32_t* forced_iters;/* host [n_steps] or NULL: run exactly this many
                                 material evaluations per step (ignores tol)   */
  double switch_tol;          /* MS_PREC_FP32_BULK: FP32 -> FP64 switch (<=0: 1e-5) */
  int stress_mask;            /* mixed boundary conditions (Sec. 3): bit c set = the
                                 macroscopic STRESS of Voigt component c is prescribed
                                 (its entry of E_k is ignored; its mean strain is solved
                                 for), e.g. 0x3e for uniaxial tension along 11; 0: all
                                 strains prescribed                                    */
  const double* Sigma;        /* host [n_steps][6] prescribed stresses or NULL (= 0) */
  int ref_update;             /* 1: at the start of every load step, adjust the
                                 reference medium to the tangents of a material
                                 evaluation at the predicted strain (Sec. 3); 0: the
                                 fixed elastic reference                               */
  int integrator;             /* 0: the implicit-Euler update (gsm_update) of every
                                 phase; 1: the force-potential form integrated over
                                 each load step by ode23 (gsm_update_ode23) from the
                                 voxel's strain at t_n to the current iterate; 2: the
                                 same by ode12 (gsm_update_ode, GSM_ODE12); 3: by
                                 ode23s (GSM_ODE23S); 1, 2 or 3 are needed for
                                 GSM_PSI_ELASTIC_VP_KIN phases; FP64 only             */
  double ode_rtol, ode_atol;  /* integrator >= 1: stress-error tolerances (rtol > 0,
                                 atol >= 0); keep them well below `tol`: an update
                                 that is not converged to better than the equilibrium
                                 tolerance stalls the fixed point                      */
  int ode_max_substeps;       /* integrator >= 1: attempts per voxel and step (>= 1)  */
} ms_load;

typedef struct ms_state {
  double* eps;                /* device [6][N^3] strain; in/out if resume     */
  double* z;                  /* device [6][N^3] internal variables (z_n)     */
  int resume;                 /* 0: start from eps = 0, z = 0, E_prev = 0;
                                 1: continue from eps, z, E_prev              */
  double E_prev[6];           /* macroscopic strain of the previous step      */
} ms_state;

typedef struct ms_result {
  double* Sigma;              /* host [n_steps][6] mean stress per step (out)  */
  int32_t* iters;             /* host [n_steps] material evaluations per step */
  double* final_error;        /* host [n_steps] e at the end of each step     */
  int32_t* fp32_iters;        /* host [n_steps] of which in FP32 (may be NULL) */
  int64_t total_iters;        /* out                                          */
  double* E;                  /* host [n_steps][6] macroscopic strain at the end of
                                 each step (may be NULL)                      */
  double* reference;          /* host [n_steps][2] (lambda0, mu0) of each step's
                                 reference medium (may be NULL)               */
} ms_result;

typedef struct ms_context* ms_handle;

/*
 * ms_create -- plan a basic-scheme solver for one problem: allocates the
 * device workspace (fields, FFT buffers, reduction scratch) and cuFFT plans
 * on the current device and binds them to `stream`.  The phase pointer and
 * the laws must stay valid until ms_destroy.  Synchronous.
 * Errors: GSM_EINVAL, GSM_ENOMEM, GSM_ECUDA.
 */
int ms_create(ms_handle* out, const ms_problem* prob, void* stream);
int ms_destroy(ms_handle h);

/* ms_workspace_bytes -- device bytes ms_create will allocate for `prob`
 * (fields, FFT buffers and cuFFT work areas); for admission control. */
size_t ms_workspace_bytes(const ms_problem* prob);

/*
 * ms_run -- solve a load history on a planned context.  `state` may be NULL
 * (fresh start, internal fields); otherwise state->eps / state->z are device
 * [6][N^3] FP64 arrays used as the solver's fields (read when resume = 1,
 * always written back).  Synchronous: reads one FP64 residual per iteration.
 * A problem with GSM_PSI_ELASTIC_VP_KIN phases keeps its seventh internal
 * variable (the accumulated plastic strain) inside the context: it starts
 * fresh only (resume = 1 gives GSM_ENOTSUP).
 * Errors: GSM_EINVAL, GSM_ECUDA, GSM_ENOTSUP (integrator 1, 2 or 3 with a precision
 * other than MS_PREC_FP64, a VP_KIN phase with integrator 0), GSM_ENOTCONV
 * (some step hit max_iter; the result is still filled in).
 */
int ms_run(ms_handle h, const ms_load* load, ms_state* state, ms_result* result);

/* ms_solve -- one-shot ms_create + ms_run + ms_destroy. */
int ms_solve(const ms_problem* prob, const ms_load* load, ms_state* state, ms_result* result, void* stream);

/* ============================================ adjoint of the load history
 *
 * Gradient of J = w . Sigma_K (the last step's mean stress) with respect to
 * the parameters (E, sigma0, n) of one Norton phase, through the whole load
 * history: material update and basic scheme, discrete adjoint with per-step
 * checkpoints (the paper's AD is local to a voxel, Sec. 4.1/5; this is its
 * continuation to the homogenization run).  Backward over the steps, each
 * step solves the adjoint equilibrium P_V(C_t lam) = P_V(a_u) with the
 * consistent tangent field C_t by conjugate gradients on G C_t lam = G a_u,
 * G the Green operator of the identity reference (the orthogonal projector
 * onto compatible zero-mean strain fields; G C_t is symmetric positive
 * definite there), in about the square root of the basic scheme's
 * iterations.  A step whose CG meets a non-positive curvature falls back to
 * the basic-scheme fixed point on the tangent field's isotropic reference.
 */
typedef struct ms_tape* ms_tape_handle;

/* ms_run_taped -- ms_run from a fresh state (no resume) that keeps the
 * checkpoints (eps_k, z_{k-1}) of every step on the device (2 * 6 * N^3
 * doubles per step) plus adjoint work arrays (71 * N^3 doubles).  The tape
 * refers to the context, which must outlive it.  Prescribed macroscopic
 * strains and the implicit-Euler update only (stress_mask = 0, integrator =
 * 0; GSM_ENOTSUP otherwise); the reference medium may be fixed or per step
 * (ref_update), which changes the iteration counts, not the converged states
 * the adjoint linearises.  Errors as ms_run. */
int ms_run_taped(ms_handle h, const ms_load* load, ms_result* result, ms_tape_handle* tape);

/* ms_adjoint -- dJ/d(E, sigma0, n) of the Norton phase `phase_id` for the
 * weights w (host [6], tensor-shear Voigt pairing with Sigma_K) into grad
 * (host [3]).  Each adjoint equilibrium is solved until its residual falls
 * by `tol`, at most max_iter iterations (lam_iters: host [n_steps] or NULL,
 * the iterations each step took: CG iterations, or fixed-point evaluations
 * where a step fell back).  Synchronous.  Returns GSM_ENOTCONV, with
 * grad filled, when a step reached max_iter.  Errors: GSM_EINVAL, GSM_ECUDA. */
int ms_adjoint(ms_tape_handle tape, const double* w, int phase_id, double tol, int max_iter, double* grad,
               int32_t* lam_iters);
int ms_tape_destroy(ms_tape_handle tape);

/* ===================================================== serving (batched jobs)
 *
 * A server keeps many basic-scheme jobs resident on one GPU and advances the
 * active jobs by one iteration per serve_tick: one material launch, one
 * Green-operator launch and one reduction launch cover every job of the tick
 * (per-job cuFFT calls in between), then one device-to-host copy of their
 * errors.  Jobs that arrive while others run are admitted first come first
 * served at the next tick when a slot (max_active) and the HBM budget allow;
 * finished jobs release their memory at once.  Which active jobs a tick takes
 * is fair share: each job carries the GPU work it has received (N^3 per FP32
 * iteration, 8 N^3 per FP64 one) and a tick takes the jobs within one
 * largest-job iteration of the least-served one, so a small grid runs many
 * iterations while a large one runs one; an admitted job starts at the
 * least-served active job's count.  A job's arithmetic does not depend on
 * the other jobs or on the schedule: its results are bit-identical alone or
 * in a mix.
 * (The paper has no serving layer; this is the continuous-batching engine
 * around its material law and basic scheme.)
 */

typedef struct serve_job {
  int N;                      /* grid size, 2 <= N <= 1024                    */
  const uint8_t* phase;       /* HOST [N^3] phase ids (copied at submission)  */
  int n_phases;               /* 1 .. 16                                      */
  const gsm_handle* laws;     /* host [n_phases] (copied at submission)       */
  int precision;              /* MS_PREC_*                                    */
  int n_steps;                /* load history, as in ms_load                  */
  const double* E;            /* host [n_steps][6]                            */
  const double* h;            /* host [n_steps]                               */
  double tol;
  int max_iter;
  double switch_tol;          /* <= 0: 1e-5                                   */
  int integrator;             /* as ms_load.integrator: 0 implicit Euler, 1 ode23,
                                 2 ode12, 3 ode23s (1-3 with MS_PREC_FP64 only;
                                 needed for GSM_PSI_ELASTIC_VP_KIN phases)     */
  double ode_rtol, ode_atol;  /* integrator >= 1, as in ms_load                */
  int ode_max_substeps;       /* integrator >= 1, as in ms_load                */
} serve_job;

typedef struct serve_server* serve_handle;

/* serve_create -- server with an HBM budget (bytes for job fields, work areas
 * and cuFFT plans) and at most max_active (1..256) jobs per tick, on `stream`.
 * Errors: GSM_EINVAL, GSM_ENOMEM. */
int serve_create(serve_handle* out, size_t hbm_budget_bytes, int max_active, void* stream);
int serve_destroy(serve_handle h);

/* serve_submit -- queue a job (host copies of all inputs; the caller's arrays
 * may be freed on return) and return its id.  Jobs with ODE-integrated laws
 * are batched with the others (their own launch group per integrator) and
 * also take the ODE work arrays from the budget (8 N^3 doubles: the strain at
 * t_n, and alpha twice for Michel-Suquet phases).  GSM_ENOMEM if the job alone
 * exceeds the budget, GSM_EINVAL on bad input, GSM_ENOTSUP for combinations
 * ms_run refuses. */
int serve_submit(serve_handle h, const serve_job* job, int64_t* id);

/* serve_tick -- admit queued jobs, run one iteration of the active jobs the
 * fair-share rule selects (at least one), retire finished ones.  Synchronous (one device-to-host copy per tick).
 * Outputs (may be NULL): active, queued and finished-but-unfetched counts. */
int serve_tick(serve_handle h, int32_t* n_active, int32_t* n_queued, int32_t* n_finished);

/* serve_job_state -- 0 queued, 1 active, 2 done, 3 done with a step at
 * max_iter; also the current step and the material evaluations so far. */
int serve_job_state(serve_handle h, int64_t id, int32_t* state, int32_t* step, int64_t* total_iters);

/* serve_fetch -- results of a finished job (host [n_steps][6] Sigma,
 * [n_steps] iterations and final errors); forgets the job.  Returns
 * GSM_ENOTCONV if a step hit max_iter, GSM_EINVAL if not finished. */
int serve_fetch(serve_handle h, int64_t id, double* Sigma, int32_t* iters, double* final_error);

/* serve_job_bytes -- device bytes a job of this size takes from the budget
 * (fields, work areas, and its cuFFT plans if none of that size exist yet;
 * jobs with ODE-integrated laws add their ODE work arrays). */
size_t serve_job_bytes(int N, int precision);

/*
 * ms_evaluate_noalloc -- one FP64 material evaluation of an N^3 phase field
 * and its FP64 mean stress, without allocating anything.  The paper has no
 * counterpart: this entry point exists for callers that cannot call
 * cudaMalloc (a process whose device memory belongs to another allocator, or
 * code that must not allocate or synchronise while it runs).
 *   N        grid size, 2 <= N <= 1024 (larger N returns GSM_EINVAL)
 *   phase    device [N^3] phase ids < n_phases (1 <= n_phases <= 16)
 *   laws     host [n_phases] materials
 *   eps      device [6][N^3] strain (normalised, engineering shears)   (in)
 *   z_n      device [6][N^3] internal variables at t_n                  (in)
 *   sigma    device [6][N^3] stress                                     (out)
 *   z        device [6][N^3] internal variables at t_{n+1}; 0 in elastic phases (out)
 *   mean     device [6] FP64 mean of sigma                              (out)
 * Same kernel and reduction as the material step of ms_run.  Its scratch is
 * a file-scope device array of 6*1024+8 doubles (the per-block partial sums
 * and the reduced result) that every GPU loading the library holds until
 * exit, so the material launch always uses at most 1024 blocks, which loop
 * over the voxels; the N <= 1024 bound is the input limit of every grid
 * entry point, not a consequence of that cap.  All calls share the array, so
 * calls whose work overlaps on the GPU race.  The first call on a device
 * looks up the array's device address (cudaGetSymbolAddress) and the
 * kernel's occupancy, under a lock: make that first call before any stream
 * capture.  Asynchronous on `stream`.  Errors: GSM_EINVAL, GSM_ECUDA.
 */
int ms_evaluate_noalloc(int N, const uint8_t* phase, int n_phases, const gsm_handle* laws, double step_h,
                        const double* eps, const double* z_n, double* sigma, double* z, double* mean, void* stream);

#ifdef __cplusplus
}
#endif

#endif /* GSM_GB300_H */
