/*
 * fcns.h -- C ABI of the GB300 FC-Gram Navier-Stokes library (libfcns.so).
 *
 * Method: Fontana, Bruno, Mininni, Dmitruk, "Fourier continuation method for
 * incompressible fluids with boundaries" (FC-Gram pseudospectral
 * Navier-Stokes in a cuboid with walls at z = 0, Lz and periodic x, y).
 *
 * Conventions shared by every entry point:
 *   - Every call returns an fc_status; no C++ exception crosses the ABI.
 *   - Arguments are validated synchronously: FC_ERR_ARG for bad values or
 *     NULL pointers, FC_ERR_UNSUPPORTED for sizes outside what the compiled
 *     kernels cover.  A failing call writes nothing.
 *   - "Device pointer" arguments are caller-owned CUDA device allocations
 *     (for example PyTorch tensors), contiguous, 16-byte aligned, on the
 *     current CUDA device.  "Host pointer" arguments are ordinary host memory.
 *   - Kernels are enqueued on the caller's stream (fc_stream_t is a
 *     cudaStream_t; NULL means the legacy default stream) and the calls
 *     return without synchronising unless stated otherwise.  Asynchronous
 *     CUDA failures surface as FC_ERR_CUDA from the next call that checks.
 *   - Physical fields are row-major [nf][Nz][Ny][Nx] real (float or double),
 *     x fastest.  The simulation state (see ns_get_state) is internal.
 *   - Grids include both walls: z_s = s Lz/(Nz-1), s = 0..Nz-1; the
 *     continued (periodic) grid has N' = Nz + C points and period
 *     L'z = N' Lz/(Nz-1).  Forward transforms are unnormalised, inverse
 *     transforms carry 1/N.
 */
#ifndef FCNS_H
#define FCNS_H

#include <stddef.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
  FC_OK = 0,
  FC_ERR_ARG = 1,          /* invalid argument or NULL pointer                    */
  FC_ERR_UNSUPPORTED = 2,  /* size outside the compiled kernel set                 */
  FC_ERR_CUDA = 3,         /* a CUDA runtime call or kernel launch failed          */
  FC_ERR_NOMEM = 4,        /* device or host allocation failed / workspace too small */
  FC_ERR_TIMEOUT = 5,      /* a bounded device wait gave up                        */
  FC_ERR_NONFINITE = 6,    /* non-finite values detected in an output             */
  FC_ERR_STATE = 7         /* call not valid in the object's current state         */
} fc_status;

typedef enum { FC_F32 = 0, FC_F64 = 1 } fc_dtype;

typedef struct fc_plan* fc_plan_t;
typedef struct ns_sim* ns_sim_t;
typedef void* fc_stream_t; /* cudaStream_t */

/* Human-readable name of a status code (static string, never NULL). */
const char* fc_status_str(fc_status s);

/* Text of the last error detected on the calling thread (static per thread). */
const char* fc_last_error(void);

/* ------------------------------------------------------------------------ */
/* FC-Gram continuation plan                                                  */
/* ------------------------------------------------------------------------ */

/*
 * fc_setup -- build the FC-Gram continuation tables for d matching points and
 * C continuation points (Sec. 3, continuation formula; App. B, Gram basis by
 * QR of the Vandermonde matrix on the d matching points and oversampled
 * least-squares Fourier continuations of each Gram polynomial with
 * periodicity interval [1 - delta_r, 2b - (1 - delta_r)]).  Host only; the
 * tables are computed in binary128 (_Float128) for d <= 5 and in
 * double-binary128 (about 67 digits) for d >= 6, whose fits -- e.g. the
 * paper's d = 7, C = 33 -- are too ill-conditioned for 34 digits, and rounded
 * to double.
 *   d   number of matching points, 2 <= d <= 10.
 *   C   number of continuation points, d <= C <= 64.
 *   Nz  number of physical z points including both walls, Nz >= 2 d.
 *   out receives a new plan (owned by the caller, release with fc_destroy).
 * Uses the bandwidth M = floor(2 (d + C) / 3) and oversampling 20.
 * Device tables are created lazily, once per device, by the first call that
 * needs them on that device (that first call allocates and must not be
 * inside a CUDA graph capture).
 */
fc_status fc_setup(int d, int C, int Nz, fc_plan_t* out);

/* As fc_setup with an explicit trigonometric bandwidth M (number of cosine /
 * sine pairs, 1 <= M) and oversampling factor n_os (>= 1). */
fc_status fc_setup_ex(int d, int C, int Nz, int M, int n_os, fc_plan_t* out);

/* Copy the right-end continuation matrix M_r = A_r Q_r^T (C rows x d
 * columns, row-major) to host memory Mr_out (C*d doubles).  Row j gives the
 * weights of the last d samples f_{Nz-d..Nz-1} for continuation point
 * Nz + j.  The left-end matrix is its row/column reversal (Sec. 3). */
fc_status fc_plan_matrix(fc_plan_t plan, double* Mr_out);

/* Sizes of a plan (any output pointer may be NULL); ls_residual is the
 * largest relative least-squares residual of the continuation fits. */
fc_status fc_plan_info(fc_plan_t plan, int* d, int* C, int* Nz, int* M, int* n_os,
                       double* ls_residual);

/* Release a plan and its device tables (synchronises the devices it used). */
fc_status fc_destroy(fc_plan_t plan);

/*
 * fc_deriv_z -- first and/or second z-derivative of real fields by FC-Gram
 * (Sec. 3: continuation of every z-line from its first and last d samples to
 * N' = Nz + C points; Sec. 4.2: multiplication of the Fourier coefficients by
 * i k (Nyquist entry zeroed) or -k^2; inverse transform truncated to the Nz
 * physical points).  The continuation product is evaluated in double (in the
 * float32 path with compensated float-float arithmetic of double accuracy).
 *   dtype  FC_F32: f, df, d2f are float; FC_F64: double.
 *   batch, Nx, Ny  field count and horizontal sizes (each >= 1); the line
 *          count batch*Nx*Ny must stay below 2^31.
 *   Lz     domain height (> 0); dz = Lz/(Nz-1).
 *   f      device pointer, [batch][Nz][Ny][Nx].
 *   df     device pointer for d f/dz, same layout, or NULL.
 *   d2f    device pointer for d^2 f/dz^2, same layout, or NULL.
 *          At least one of df, d2f must be non-NULL; outputs must not
 *          overlap f.
 *   stream CUDA stream for the launch.
 * Needs no workspace.  Transform length: N' itself when it is a compiled
 * smooth length (64, 128, 256, 512, 768, 1024, 1536), else the smallest
 * compiled length >= N' + Nz - 1 (up to 1536); FC_ERR_UNSUPPORTED when
 * neither exists.
 */
fc_status fc_deriv_z(fc_plan_t plan, fc_dtype dtype, int batch, int Nx, int Ny, double Lz,
                     const void* f, void* df, void* d2f, fc_stream_t stream);

/*
 * fc_deriv_z_noalloc -- the same computation and arguments as fc_deriv_z,
 * for callers that cannot let the library allocate device memory:
 * applications whose device memory belongs to a host framework or to a
 * fixed-size arena and that forbid allocations by plug-ins, and programs
 * running under a device-memory budget that a library must not grow.
 * (fc_deriv_z allocates its tables with cudaMalloc on the first call of a
 * plan on a device.)  The paper has no counterpart; this is a deployment
 * variant of fc_deriv_z, and its results are bitwise those of fc_deriv_z.
 *   - Calls no cudaMalloc, cudaFree or other allocating routine.  The plan's
 *     tables (continuation matrix, kernel spectra, twiddles) live in one
 *     fixed 128 KiB static device array that every GPU loading the library
 *     reserves until the process exits.
 *   - The first call on each device looks up that array's device address
 *     (cudaGetSymbolAddress) with the device current and keeps it for the
 *     life of the process: resetting the device (cudaDeviceReset) after that
 *     first call is not supported.
 *   - When the plan or the precision differs from those of the previous call
 *     on the device, the call first copies the plan's tables into the array
 *     on `stream` from the plan's (pageable) host memory; such a copy waits
 *     for the work already queued on `stream` before the call returns.  A
 *     call with the same plan and precision as the previous call on the
 *     device copies nothing and only enqueues the kernel.
 *   - Every call shares the array and the tables stay there after the call:
 *     calls whose copies and kernels can overlap on the GPU (on other
 *     streams, from other host threads) race on it and must be serialised by
 *     the caller.
 *   - A plan whose tables would not fit the 128 KiB array returns
 *     FC_ERR_UNSUPPORTED (the tables of every compiled transform length fit:
 *     at most 100 KiB, float64 at length 1536); arguments are checked as in
 *     fc_deriv_z.
 */
fc_status fc_deriv_z_noalloc(fc_plan_t plan, fc_dtype dtype, int batch, int Nx, int Ny, double Lz,
                             const void* f, void* df, void* d2f, fc_stream_t stream);

/*
 * fc_deriv_z_host -- the computation of fc_deriv_z on HOST arrays f, df, d2f
 * (same layout [batch][Nz][Ny][Nx] and arguments; df or d2f may be NULL).
 * The library moves slabs of y rows (all z and x of a field, at most about
 * 256 MB of input each, an even number of rows, the slabs of a field of
 * nearly equal size; the first slab of a call about a quarter of that, so
 * that the device-to-host copies start sooner) through three rotating device
 * buffers
 * on three internal streams: the host-to-device copy of one slab, the kernel
 * of the previous one and the device-to-host copies of the one before run
 * concurrently.  Results are bitwise those of fc_deriv_z on device copies of
 * the same arrays.  Synchronous: it starts after the work already queued on
 * `stream` and returns when the outputs are in host memory.  Host arrays
 * should be page-locked (cudaHostAlloc / cudaHostRegister) for the copies to
 * overlap; pageable arrays work at the driver's staged-copy speed.  The
 * staging buffers (3 x 3 slabs) stay allocated with the plan, per device,
 * until fc_destroy; calls on one plan run one at a time.
 */
fc_status fc_deriv_z_host(fc_plan_t plan, fc_dtype dtype, int batch, int Nx, int Ny, double Lz,
                          const void* f, void* df, void* d2f, fc_stream_t stream);

/* fc_deriv_z_host with the slab size in bytes of input chosen by the caller
 * (at least two y rows are moved at a time). */
fc_status fc_deriv_z_host_ex(fc_plan_t plan, fc_dtype dtype, int batch, int Nx, int Ny, double Lz,
                             const void* f, void* df, void* d2f, size_t slab_bytes, fc_stream_t stream);

/* ------------------------------------------------------------------------ */
/* Navier-Stokes / Boussinesq simulation                                     */
/* ------------------------------------------------------------------------ */

typedef struct {
  int Nx, Ny, Nz;        /* physical grid; Nx, Ny even, Nz >= 2 d                  */
  int d, C;              /* FC-Gram matching / continuation points                  */
  int nfields;           /* 3: Navier-Stokes (u, v, w); 4: Boussinesq (+ theta)     */
  int rk_order;          /* o of the time-splitting low-storage RK (1..4)           */
  double Lx, Ly, Lz;     /* box size                                                */
  double nu, kappa;      /* viscosity, thermal diffusivity                          */
  double gamma;          /* Boussinesq coupling (Sec. 7); unused for nfields = 3    */
  double forcing_x;      /* constant mean-pressure forcing +F x_hat (Sec. 6)        */
  int filter;            /* 0: exponential filter in x, y, z (Sec. 4.3);
                            1: sharp 2/3 mask in x, y and exponential in z          */
  double filter_beta;    /* beta (16 ln 10 for double precision digits)            */
  double filter_2p;      /* 2p (100)                                                */
  fc_dtype prec;         /* FC_F32: float transforms and products with the
                            continuation products, the homogeneous-pressure
                            coefficients and the mean-flow line in double;
                            FC_F64: everything in double                           */
} ns_params;

/* Fill *p with the defaults: d = 5, C = 25, nfields = 3, rk_order = 3,
 * Lx = Ly = 2 pi, Lz = 1, nu = 1e-2, kappa = gamma = forcing_x = 0,
 * filter = 1, filter_beta = 16 ln 10, filter_2p = 100, prec = FC_F64.
 * Nx, Ny, Nz are set to 0 and must be filled in. */
fc_status ns_params_default(ns_params* p);

/* Device workspace (bytes) that ns_create needs for these parameters. */
fc_status ns_workspace_bytes(const ns_params* p, size_t* bytes);

/*
 * ns_create -- create a simulation object holding the state of the
 * nfields fields, the wall pressure-gradient planes (Sec. 4.4 step 2) and the
 * tables.  dev_workspace (device pointer, >= ns_workspace_bytes) is used for
 * every device buffer; if it is NULL the library allocates it itself with
 * cudaMalloc and frees it in ns_destroy.  Creation uploads tables with
 * synchronous copies on the current device.
 * z transforms: when N' = Nz + C is itself a compiled length (64, 128, 256,
 * 512, 768, 1024, 1536 -- the paper's choice of smooth N') the z derivatives and
 * filter are length-N' spectral multipliers and the projection's DFTs plain
 * length-N' transforms; otherwise they are circular convolutions and
 * Bluestein DFTs on a padded length L >= max(N' + Nz - 1, 2 N' - 1) (160,
 * 288, 320, 576, 1080 or 1152).  FC_ERR_UNSUPPORTED when no compiled length fits,
 * Nx or Ny is not one of 16, 32, 64, 96, 128, 192, 256, 512, 1024, or, in
 * double precision, L > 576 or Nx > 512.
 */
fc_status ns_create(const ns_params* p, void* dev_workspace, size_t bytes, ns_sim_t* out);

/* Release the object (synchronises its device). */
fc_status ns_destroy(ns_sim_t sim);

/* Set the state from physical fields phys (device pointer,
 * [nf][Nz][Ny][Nx] in the simulation's precision): the state becomes the
 * FC continuation of phys in (kx, ky, z') (Sec. 3), and the wall
 * pressure-gradient planes are reset to zero. */
fc_status ns_set_fields(ns_sim_t sim, const void* phys, fc_stream_t stream);

/* Physical fields of the current state (first Nz points of the inverse
 * transforms), device pointer [nf][Nz][Ny][Nx]. */
fc_status ns_get_fields(ns_sim_t sim, void* phys, fc_stream_t stream);

/* Copy the state to / from a device buffer (checkpoint / restore).  The
 * buffer holds nf * (Nz+C) * Ny * Kxp complex values of the simulation's
 * precision, Kxp = Nx/2+1 rounded up to a multiple of 16, in the library's
 * internal order: the fields in (kx, ky, z') on the continued grid, lines
 * (ky * Kxp + kx) grouped in tiles of 16 whose z' rows are contiguous.  A
 * length-(Nz+C) DFT along z' turns it into the continued spectral field of
 * the paper. */
fc_status ns_get_state(ns_sim_t sim, void* spec, fc_stream_t stream);
fc_status ns_put_state(ns_sim_t sim, const void* spec, fc_stream_t stream);

/* Wall pressure-gradient planes: [2 walls][2 components][Ny][Nx/2+1] complex
 * double, device pointer (get copies out, put copies in). */
fc_status ns_get_wall_gradp(ns_sim_t sim, void* gradp, fc_stream_t stream);
fc_status ns_put_wall_gradp(ns_sim_t sim, const void* gradp, fc_stream_t stream);

/*
 * ns_rhs -- right-hand side of the pressureless momentum (and temperature)
 * equations for the physical fields phys_in (Sec. 4.2 and Sec. 4.4 step 1):
 * with v^c the FC continuation of phys_in,
 *   rhs = filter[ -(v.grad)v + F x_hat (+ gamma theta z_hat) ] - nu k^2 v^c
 * (theta: filter[ -(v.grad)theta + gamma w ] - kappa k^2 theta^c),
 * returned at the Nz physical points.  Overwrites the simulation's working
 * buffers (not its state).  phys_in, rhs_out: device pointers
 * [nf][Nz][Ny][Nx].
 */
fc_status ns_rhs(ns_sim_t sim, const void* phys_in, void* rhs_out, fc_stream_t stream);

/*
 * fc_poisson_project -- pressure solve and projection of a physical
 * pressureless velocity v* (Sec. 4.1-4.2, Sec. 4.4 steps 2-5) with the
 * readings phi = dt_stage p:
 *   inject v*_par = dt_stage grad_par p_prev at z = 0, Lz (p_prev: the
 *   simulation's wall planes), FC-continue, grad phi^I = k (k.v*)/k^2,
 *   b, t = w* - d_z phi^I at the walls, homogeneous solution
 *   A e^{g(z-Lz)} + B e^{-g z} (+ D z for the mean mode, D = (b+t)/2),
 *   v = v* - grad phi^I - grad phi^H, and stores grad_par p = grad_par phi /
 *   dt_stage at the walls as the simulation's new wall planes.
 *   vstar_phys, v_phys  device pointers [3][Nz][Ny][Nx] (velocity only).
 *   gradp_wall          device pointer for a copy of the new wall planes
 *                       ([2][2][Ny][Nx/2+1] complex double) or NULL.
 * Leaves the simulation's state unchanged (its work buffers are overwritten).
 */
fc_status fc_poisson_project(ns_sim_t sim, double dt_stage, const void* vstar_phys, void* v_phys,
                             void* gradp_wall, fc_stream_t stream);

/*
 * rk_step -- advance the state by one time step dt with the time-splitting
 * low-storage Runge-Kutta scheme of order rk_order (Sec. 4.4), stage steps
 * dt_j = dt / (o + 1 - j).
 */
fc_status rk_step(ns_sim_t sim, double dt, fc_stream_t stream);

/*
 * ns_diagnostics -- scalar diagnostics of the current state, synchronous
 * (host outputs; any pointer may be NULL):
 *   div_ms       mean square of div v over the physical grid points, with the
 *                FC z-derivative and spectral x, y derivatives (Sec. 6),
 *   wall_u_ms    mean square of u over the points of both walls,
 *   wall_w_ms    the same for w (zero to round-off after a projection),
 *   flow_rate    mean of u over the physical grid points,
 *   nusselt      (Nu at z = 0 + Nu at z = Lz)/2 with Nu = 1 - <d_z theta>/gamma
 *                (Sec. 7; 0 for nfields = 3).
 * Overwrites the simulation's work buffers (not its state).
 */
fc_status ns_diagnostics(ns_sim_t sim, double* div_ms, double* wall_u_ms, double* wall_w_ms,
                         double* flow_rate, double* nusselt, fc_stream_t stream);

/*
 * ns_set_diag_series -- time series of the ns_diagnostics quantities (the
 * flow-rate and Nusselt-number histories of Sec. 6 and 7) kept on the
 * device: after every `every`-th rk_step the diagnostic sums of the new state
 * are computed on the step's stream into the next of 4096 device slots, with
 * no synchronisation and no host copy (recording stops when the slots are
 * full).  every = 0 stops recording.  Every call clears the series and
 * restarts the step count.  ns_batch_step does not record.  FC_ERR_ARG for
 * every < 0.  Each recorded step costs one z-derivative pass and one
 * reduction (as ns_diagnostics) and overwrites the work buffers.
 */
fc_status ns_set_diag_series(ns_sim_t sim, int every);

/*
 * ns_get_diag_series -- copy the first min(max, recorded) entries of the
 * series to host memory, synchronously (the copy is enqueued on `stream`,
 * which must be the stream of the recorded steps or ordered after them):
 * values[5 i + 0 .. 4] = div_ms, wall_u_ms, wall_w_ms, flow_rate, nusselt of
 * entry i (the definitions and normalisation of ns_diagnostics: the values
 * ns_diagnostics returns for that state, up to the order of the float64
 * atomic additions of the reduction); steps[i] (may be
 * NULL) = its step number counted from ns_set_diag_series; *count (may be
 * NULL) = the number of entries recorded.  FC_ERR_ARG for max < 0 or a NULL
 * values with max > 0.
 */
fc_status ns_get_diag_series(ns_sim_t sim, int max, double* values, long long* steps, int* count,
                             fc_stream_t stream);

/*
 * ns_profiles -- horizontal statistics of the current state (Sec. 6 r.m.s.
 * velocity profiles and spectra; Sec. 7 temperature profiles), synchronous,
 * host outputs (each may be NULL), by Parseval from the state's physical rows:
 *   mean[f*Nz + s]       <q_f>_{x,y} at z_s,
 *   rms[f*Nz + s]        sqrt(<(q_f - <q_f>_{x,y})^2>_{x,y}) at z_s,
 *   spectrum[f*ns + j]   (1/Lz) int dz of the horizontal power of q_f in shell j
 *                        (modes with j - 1/2 <= |k_perp|/dk < j + 1/2, the mean
 *                        mode excluded; trapezoid rule over the Nz levels), so
 *                        sum_j spectrum = <rms^2>_z;
 * ns and dk from ns_spectrum_shells (dk = min(2 pi/Lx, 2 pi/Ly)).  Uses the
 * simulation's work buffers (not its state).
 */
fc_status ns_profiles(ns_sim_t sim, double* mean, double* rms, double* spectrum, fc_stream_t stream);

/* Number of spectrum shells and their width (either pointer may be NULL). */
fc_status ns_spectrum_shells(ns_sim_t sim, int* nshell, double* dk);

/*
 * ns_interpolate -- restart on another grid (Sec. 6: "spectral interpolation,
 * by zero padding the transformed fields in the wavenumber domain"): the state
 * of dst becomes the interpolant of src's state, re-continued on dst's grid;
 * dst's wall planes are reset to zero.  x, y: zero padding (dst Nx >= src Nx,
 * dst Ny >= src Ny), coefficients scaled by (Nx2 Ny2)/(Nx1 Ny1), a coarse
 * Nyquist coefficient split in half between +N/2 and -N/2.  z: the
 * N'-periodic series of each source line (Nyquist term as a cosine) evaluated
 * at dst's Nz physical points (any Nz; the continuation period changes with
 * the grid, so z coefficients are not padded directly).  Both simulations on
 * the current device, same box, nfields and precision (else FC_ERR_ARG);
 * FC_ERR_UNSUPPORTED if dst's work buffers cannot hold the Nz x N'(src)
 * weight table.  Uploads the weights with a synchronous copy.
 */
fc_status ns_interpolate(ns_sim_t dst, ns_sim_t src, fc_stream_t stream);

/*
 * Initial perturbation (App. A): a random solenoidal velocity that vanishes
 * at both walls, built from curl eigenfunctions,
 *   q = curl curl(phi z_hat) + curl(psi z_hat),
 *   phi = sum a e^{i(kx x + ky y)} g_m(z'),  psi = sum b e^{i(kx x + ky y)} sin(m pi (z' + 1/2)),
 * z' = z/Lz - 1/2, g_m the Chandrasekhar-Reid functions
 * (cosh(l z')/cosh(l/2) - cos(l z')/cos(l/2) for odd m, sinh / sin for even
 * m, l = lambda_m, the m-th root of g_m'(+-1/2) = 0), a = k^slope_phi
 * e^{2 pi i u_a}, b = k^slope_psi e^{2 pi i u_b}, k^2 = kx^2 + ky^2 +
 * lambda_m^2, kx = 2 pi n / Lx, ky = 2 pi l / Ly.  Modes: the half plane
 * (l > 0, or l = 0 and n > 0) of the annulus kperp2_min <= kx^2 + ky^2 <=
 * kperp2_max (inclusive within a relative 1e-12), and m_min <= m <= m_max;
 * the real part is taken.  App. A's choice is the default: annulus [4, 25],
 * m = 2..5, slopes -4 and -3.
 */
typedef struct {
  double Lx, Ly, Lz;               /* x, y periods; wall distance (z in [0, Lz])        */
  double kperp2_min, kperp2_max;   /* annulus of kx^2 + ky^2                            */
  int m_min, m_max;                /* vertical indices, 1 <= m_min <= m_max <= 64       */
  double slope_phi, slope_psi;     /* exponents of |a| and |b| in k                     */
  double amplitude;                /* largest component magnitude of the result         */
} fc_noise_params;

/* The defaults above (Lx = Ly = 2 pi, Lz = 1, amplitude 1). */
fc_status fc_noise_params_default(fc_noise_params* p);

/* Number of (n, l, m) modes of these parameters (host only; the caller
 * supplies two uniform draws per mode to fc_noise).  FC_ERR_ARG for invalid
 * parameters (see fc_noise). */
fc_status fc_noise_modes(const fc_noise_params* p, int* count);

/*
 * fc_noise -- the perturbation on the grid x_i = i Lx/Nx, y_j = j Ly/Ny,
 * z_s = s Lz/(Nz - 1), written to `out` (device, [3][Nz][Ny][Nx] contiguous,
 * components u, v, w, dtype FC_F32 or FC_F64; the arithmetic is float64 in
 * both cases), scaled so that its largest component magnitude equals
 * p->amplitude.  draws: host array of ndraws = 2 x fc_noise_modes() numbers
 * in [0, 1): (u_a, u_b) per mode, modes ordered by n ascending, then l
 * ascending, then m ascending.  lambda_m and the mode amplitudes are computed
 * on the host; the profiles, the synthesis and the scaling run on the device
 * on `stream` (scratch taken with cudaMallocAsync / cudaFreeAsync on it).
 * Asynchronous with respect to the host (the draws are read before return).
 * The result is exactly solenoidal and no-slip as a function; on the grid
 * the walls hold zero to rounding.  Add it to a base flow and pass the sum to
 * ns_set_fields.  FC_ERR_ARG: invalid parameters (Lx, Ly, Lz <= 0,
 * kperp2_min > kperp2_max, m outside 1..64, non-finite values), no mode in
 * the annulus, ndraws wrong, a non-finite draw, NULL pointers, Nx <= 2 max|n|
 * or Ny <= 2 max l (a mode the grid cannot resolve), Nz < 2;
 * FC_ERR_UNSUPPORTED for more than 511 kx indices on each side of the annulus
 * (max |n| > 511); FC_ERR_NOMEM if the scratch cannot be allocated.
 */
fc_status fc_noise(const fc_noise_params* p, fc_dtype dtype, int Nx, int Ny, int Nz, const double* draws,
                   int ndraws, void* out, fc_stream_t stream);

/*
 * ns_tune -- kernel variants of the five kernel kinds of the RK step (z
 * derivatives, stage combine, projection, y inverse, y forward).  Per kind,
 * bit 0 selects the lines per CTA (tile): two sizes of each kind are
 * compiled.  For the three z kinds of a float32 simulation whose padded z
 * length has a second radix schedule compiled (L = 160, 288, 320: the two
 * factors of the two-pass length-L transform swapped, e.g. 288 = 16 x 18 or
 * 18 x 16), bit 1 selects that schedule.  mode 0: the built-in defaults
 * (all 0); 1: autotune -- time every variant of each kernel on this
 * simulation's buffers and keep the fastest (synchronous; cached per process
 * and size; the state and the wall planes are preserved); 2: set from tiles
 * (bits a kind does not have are ignored).  tiles: 5 ints, read for mode 2,
 * written with the choice if non-NULL.  The tile does not change any result
 * (every line is computed the same way whatever the tile); the radix
 * schedule changes the rounding of the float32 transforms only (the same
 * DFTs, summed in another order).
 */
fc_status ns_tune(ns_sim_t sim, int mode, int* tiles, fc_stream_t stream);

/* ------------------------------------------------------------------------ */
/* Batched ensemble: many independent simulations, one graph launch per step */
/* ------------------------------------------------------------------------ */

typedef struct ns_batch* ns_batch_t;

/*
 * ns_batch_create -- group n simulations (created on the current device,
 * each at most once; any sizes, precisions and parameters) so that one RK
 * step of all of them (Sec. 4.4, as rk_step) runs as a single CUDA graph
 * launch.  Autotunes the tiles and radix schedules of every member first
 * (ns_tune mode 1).  The members stay owned by the caller and must outlive the batch;
 * the batch copies the array of handles.  FC_ERR_ARG for NULL / repeated
 * members, FC_ERR_STATE for members of another device.
 */
fc_status ns_batch_create(ns_sim_t* sims, int n, ns_batch_t* out);

/*
 * ns_batch_step -- advance member i by one RK step of size dt[i] (host array
 * of n positive values).  The first call for a given set of step sizes and
 * buffer rotation captures the members' kernels into a graph (members spread
 * over 8 concurrent branches) on private streams; later calls replay it with
 * one cudaGraphLaunch on `stream`.  Results are bitwise those of rk_step on
 * each member.  Up to 6 graphs are cached; members must not be stepped
 * through other calls concurrently.
 */
fc_status ns_batch_step(ns_batch_t batch, const double* dt, fc_stream_t stream);

/* Members, nodes of the last captured graph, graphs cached (NULL to skip). */
fc_status ns_batch_info(ns_batch_t batch, int* members, int* graph_nodes, int* graphs_cached);

/* Release the graphs and streams (not the members). */
fc_status ns_batch_destroy(ns_batch_t batch);

/* ------------------------------------------------------------------------ */
/* Failure detection and injection                                            */
/* ------------------------------------------------------------------------ */

/*
 * fc_count_nonfinite -- number of Inf / NaN values among n reals of type
 * dtype at the device pointer data (for example an fc_deriv_z output),
 * counted by a kernel on `stream`; synchronous (waits for the stream).
 * *count (host) receives the number; returns FC_ERR_NONFINITE when it is
 * positive, FC_OK otherwise.  n = 0 is allowed (count 0, nothing launched).
 */
fc_status fc_count_nonfinite(fc_dtype dtype, const void* data, long long n, long long* count,
                             fc_stream_t stream);

/*
 * ns_check_finite -- number of Inf / NaN values (real and imaginary parts
 * counted separately) in the simulation's state: every field on the N'
 * continued rows of every physical (kx, ky) line.  Synchronous; *count (host)
 * receives the number; FC_ERR_NONFINITE when it is positive.  Also resets
 * the flag of ns_set_finite_check to this count.
 */
fc_status ns_check_finite(ns_sim_t sim, long long* count, fc_stream_t stream);

/*
 * ns_set_finite_check -- check the state for non-finite values after every
 * `every`-th rk_step (and after every ns_batch_step of a batch holding the
 * simulation); 0 (the default) turns the check off.  The check is a kernel
 * that adds the count to a device-side flag, followed by an asynchronous
 * copy of the flag into pinned host memory, so no call waits for it: once
 * the copy of a failed check has landed, rk_step and ns_batch_step return
 * FC_ERR_NONFINITE without enqueuing work, until ns_check_finite finds the
 * state clean again (after ns_set_fields or ns_put_state).  Costs one read
 * of the state per checked step.
 */
fc_status ns_set_finite_check(ns_sim_t sim, int every);

/*
 * fc_inject_failure -- testing aid for callers' error handling, host only:
 * after `skip` further calls of the entry point named `entry` (its C name;
 * "fc_setup" covers fc_setup_ex too; "*" matches every entry point that
 * checks), the next `count` calls (count < 0: all later calls) return
 * `status` at once, enqueue nothing, write nothing and set fc_last_error to
 * "<entry>: injected failure".  entry = NULL removes every rule.  Rules can
 * also come from the environment variable FCNS_INJECT, a comma-separated
 * list of "entry:status:skip:count" (status by name, e.g. FC_ERR_CUDA, or
 * number), read on the first check.  The entry points that check are
 * fc_setup, fc_deriv_z, fc_deriv_z_noalloc, fc_deriv_z_host (and _ex),
 * fc_count_nonfinite, fc_noise, ns_create,
 * ns_set_fields, ns_get_fields, ns_get_state, ns_put_state, ns_rhs,
 * fc_poisson_project, rk_step, ns_diagnostics, ns_profiles, ns_interpolate,
 * ns_tune, ns_check_finite, ns_batch_create and ns_batch_step.
 * FC_ERR_ARG for a NULL-free rule with status FC_OK, skip < 0 or count = 0.
 */
fc_status fc_inject_failure(const char* entry, fc_status status, long long skip, long long count);

/* ------------------------------------------------------------------------ */
/* Measurement                                                                */
/* ------------------------------------------------------------------------ */

/*
 * fc_alu_probe -- arithmetic-pipe throughput probe (no counterpart in the
 * paper: it measures the float32 / float64 ceilings against which the
 * transform kernels' rooflines are stated).  Launches, on `stream`, one
 * kernel of 8 x (SM count) blocks of 256 threads, each thread running 8
 * independent chains of `iters` x 16 instructions of one kind:
 *   kind 0 FFMA (float32 fused multiply-add), 1 FADD (float32 add),
 *        2 FFMA2 (packed 2 x float32 fused multiply-add), 3 FADD2 (packed
 *        2 x float32 add), 4 DFMA (float64 fused multiply-add).
 *   iters    >= 1.
 *   sink     device pointer to 256 floats (written only in a case that
 *            cannot occur; keeps the work alive).
 *   lane_ops host pointer (may be NULL): receives the number of scalar lane
 *            operations the launch performs (two per packed instruction
 *            and thread); the caller times the launch with CUDA events.
 * Asynchronous; FC_ERR_ARG for a kind outside 0..4, iters < 1 or NULL sink.
 */
fc_status fc_alu_probe(int kind, int iters, void* sink, double* lane_ops, fc_stream_t stream);

#ifdef __cplusplus
}
#endif

#endif /* FCNS_H */
