/*
 * psatd.h - C ABI of the GB300 PSATD push library (libpsatd.so).
 *
 * The library advances Maxwell's equations with the pseudo-spectral
 * analytical time-domain (PSATD) method of arbitrary stencil order p on a
 * batch of FFT boxes, each box being a sub-domain padded with guard cells
 * ('local' decomposition, paper Fig. 1a and Sec. 1.3) or a group of
 * sub-domains with guards only on its outer faces ('hybrid' decomposition,
 * paper Fig. 1b and Sec. 2.1).  One step is, for every box:
 *   S1  3D real-to-complex FFT of E, B (and J, rho) over the padded box,
 *   S2  per-mode analytical update in k-space with order-p staggered
 *       modified wavenumbers and Yee phase shifts (Sec. 1.1),
 *   S3  inverse 3D FFT,
 * then, across boxes,
 *   S4  the guard exchange: each guard cell receives the value of the
 *       interior cell that owns the same global position (Fig. 1, step (ii)).
 *
 * Conventions shared by every entry point
 * ---------------------------------------
 *  - All pointers named "device" are CUDA device pointers of the current
 *    device; they are owned by the caller and never freed by the library.
 *  - A field component is ONE contiguous buffer holding every box of the
 *    plan, box b starting at element psatd_plan_layout(...).elem_offset.
 *    Inside a box the cell (x, y, z) is element x + n[0]*(y + n[1]*z)
 *    (x fastest).  Element type: float (precision 32) or double (64).
 *    Buffers must be at least 16-byte aligned; box offsets are multiples of
 *    64 elements.
 *  - Yee positions (in cells): E_x (i+1/2,j,k), E_y (i,j+1/2,k),
 *    E_z (i,j,k+1/2), B_x (i,j+1/2,k+1/2), B_y (i+1/2,j,k+1/2),
 *    B_z (i+1/2,j+1/2,k); J like E; rho at (i,j,k).
 *  - `stream` is a cudaStream_t passed as void* (NULL = legacy default
 *    stream).  Every device-side operation is asynchronous on it.
 *  - Errors: argument and plan errors are returned synchronously and leave
 *    no device work queued.  CUDA failures return PSATD_ERR_CUDA; the text
 *    is available from psatd_last_error.  No call aborts the process and no
 *    C++ exception crosses this boundary.
 *  - A plan is not thread-safe: use it from one host thread and one stream
 *    at a time.
 */
#ifndef PSATD_H
#define PSATD_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
  PSATD_OK = 0,
  PSATD_ERR_INVALID_ARG = 1,      /* NULL pointer, bad count, bad geometry  */
  PSATD_ERR_UNSUPPORTED_SIZE = 2, /* box size not even / not 5-smooth / too large */
  PSATD_ERR_UNSUPPORTED_ORDER = 3,/* stencil order not 0 and not even in [2, 256] */
  PSATD_ERR_OUT_OF_MEMORY = 4,    /* device allocation failed               */
  PSATD_ERR_CUDA = 5,             /* a CUDA runtime call failed             */
  PSATD_ERR_TIMEOUT = 6,          /* a bounded device-side wait ran out     */
  PSATD_ERR_STATE = 7             /* call not valid for this plan's state   */
} psatd_status;

/* Decomposition of the global domain into FFT boxes (paper Fig. 1, Sec. 2.1). */
typedef enum {
  PSATD_DECOMP_GLOBAL = 0,      /* one box, the whole periodic domain (Sec. 1.2) */
  PSATD_DECOMP_LOCAL = 1,       /* sub-domains with guards on every face (Sec. 1.3) */
  PSATD_DECOMP_HYBRID = 2,      /* groups with guards on split axes only (Sec. 2.1) */
  PSATD_DECOMP_INDEPENDENT = 3  /* self-periodic boxes: guards wrap onto own interior */
} psatd_decomp;

/* plan flags */
#define PSATD_VACUUM         0x1u /* J = rho = 0: only E and B are read and written   */
#define PSATD_RHO_CONTINUITY 0x2u /* rho is in/out, advanced by continuity; E takes   */
                                  /* its longitudinal part from Gauss's law (rho form) */
#define PSATD_J_CONSTANT     0x4u /* J is constant during each psatd_push call (the */
                                  /* time-constant current of the source workloads): */
                                  /* its spectrum is computed once per call, not per */
                                  /* step (no effect with PSATD_VACUUM)              */
#define PSATD_NO_GRAPH       0x8u /* never capture multi-step pushes in a CUDA graph   */
#define PSATD_GENERIC_KERNELS 0x10u /* diagnostics: run every box through the generic */
                                  /* kernels even where a fast path exists (the two  */
                                  /* agree to rounding)                              */
#define PSATD_PENCIL_KERNELS 0x20u /* run every box the pencil kernels accept on     */
                                  /* them (one kernel per axis pass)                 */
#define PSATD_NODAL          0x80u /* collocated variant (not in the paper, which   */
                                  /* uses staggered stencils): every component at   */
                                  /* the cell nodes, order-p centred symbol         */
                                  /* K = sum_l beta_l sin(l k h)/(l h), beta_l the  */
                                  /* Lagrange weights at 0 of the nodes l^2, no Yee */
                                  /* phase shifts                                   */
#define PSATD_PLANE_KERNELS  0x40u /* run every box the plane kernels accept on them */
                                  /* (x and y per z plane, register-resident where   */
                                  /* the shape has register codelets).  Without      */
                                  /* either flag: plane kernels when their register- */
                                  /* resident form serves every plane-eligible box,  */
                                  /* else pencil kernels; all families agree to      */
                                  /* rounding                                        */
#define PSATD_EAGER_EXCHANGE 0x100u /* store the guard cells in every step.  Without */
                                  /* it, plans whose boxes all run on the register  */
                                  /* plane kernels (or all on the pencil kernels,   */
                                  /* when each plane's guard faces form at most 3x3 */
                                  /* rectangles) defer each step's guard exchange   */
                                  /* into the next step's forward pass, which reads */
                                  /* every guard cell from the interior cell owning */
                                  /* it (the value the exchange would store), and   */
                                  /* only the last step of a push stores the guards */
                                  /* (paper Fig. 1, step (ii)); results are equal   */

/* One FFT box.  n[] counts cells including guards; each n[d] must be even,
 * 5-smooth (2^a 3^b 5^c), n[0] in [4, 1024], n[1], n[2] in [4, 512].
 * ng_lo/ng_hi are the guard widths on the low/high face of each axis
 * (0 on an axis that is periodic inside the box).  origin[] is the global
 * index of the first interior cell.  order_p is the stencil order: even in
 * [2, 256], or 0 for infinite order (pure spectral, Sec. 1.1). */
typedef struct {
  int32_t n[3];
  int32_t ng_lo[3];
  int32_t ng_hi[3];
  int64_t origin[3];
  int32_t order_p;
} psatd_box;

/* Absorbing layers (perfectly matched layers, PML).  The paper (end of its
 * Sec. 2.6) states that the solver supports the two-step PML of its
 * reference [shapoval2019two] and prints no equations; this library's
 * reading, derived from Maxwell's equations: every component is the sum of
 * two split parts, one per derivative direction (E_x = E_xy + E_xz with
 * dE_xy/dt = c^2 dB_z/dy - s_y E_xy, and so on for every component), and a
 * step is (1) the ordinary PSATD step of E and B, each split part gaining
 * the exact time integral of its derivative term over the step, then (2)
 * every split part along direction d multiplied by exp(-s_d dt).  Layers of
 * width[d] cells sit inside the global domain on both faces of axis d
 * (0: none), with conductivity s_d = sigma_max[d] (xi/width[d])^order at a
 * depth xi (cells) into the layer, evaluated at each component's Yee
 * position.  Requirements: PSATD_VACUUM (no current in the layers), not
 * PSATD_NODAL, not PSATD_DECOMP_INDEPENDENT, 0 <= width[d] <= global_n[d]/2,
 * sigma_max[d] >= 0, 0 <= order <= 16; the plan then runs the generic
 * kernels and stores the guards every step.  The plan owns one stored split
 * part per component (E_xy, E_yz, E_zx, B_xy, B_yz, B_zx; the other part is
 * the component minus it), zero at creation: start with fields that vanish
 * inside the layers, or set the parts through psatd_plan_pml_part. */
typedef struct {
  int32_t width[3];
  double sigma_max[3];
  int32_t order;
} psatd_pml;

/* Plan description.  global_n/periodic describe the global domain (ignored
 * for PSATD_DECOMP_INDEPENDENT); box interiors must tile it exactly.
 * Non-periodic axes fill guard cells outside the domain with 0.
 * dx: cell sizes; dt: time step (any sign); c: speed of light; eps0: vacuum
 * permittivity; precision: 32 (float) or 64 (double) field arithmetic (the
 * tables are always generated in double).  `boxes` is read during
 * psatd_plan_create only. */
typedef struct {
  int32_t global_n[3];
  int32_t periodic[3];
  double dx[3];
  double dt;
  double c;
  double eps0;
  int32_t precision;
  psatd_decomp decomp;
  int32_t num_boxes;
  const psatd_box* boxes;
  uint32_t flags;
  const psatd_pml* pml;   /* absorbing layers, or NULL (read during create) */
  const int32_t* tuning;  /* (knob, value) pairs ended by knob 0, at most 16
                             pairs, or NULL: PSATD_TUNE_* launch parameters
                             (read during create) */
} psatd_plan_desc;

typedef struct psatd_plan psatd_plan;

/* Field buffers (device, caller-owned, in/out). */
typedef struct {
  void* E[3];
  void* B[3];
} psatd_fields;

/* Source buffers (device, caller-owned).  J is read-only and must already
 * hold consistent guard values (fill them once with psatd_guard_exchange);
 * rho is in/out with PSATD_RHO_CONTINUITY, unused otherwise.  Pass NULL for
 * the whole struct with PSATD_VACUUM. */
typedef struct {
  const void* J[3];
  void* rho;
} psatd_sources;

/* One guard-exchange copy block (host view of the precomputed exchange
 * protocol; the paper's Sec. 2.6 computes the overlaps of its two
 * decompositions once, before the time loop, in the same way).  src_box = -1
 * means "fill with zero" (outside a non-periodic domain).  Coordinates are
 * box-local cell indices. */
typedef struct {
  int32_t dst_box, src_box;
  int32_t dst_lo[3], src_lo[3], ext[3];
} psatd_copy_block;

/* Check a description without touching the GPU.  Returns PSATD_OK or the
 * first error found; `msg` (may be NULL) receives a NUL-terminated reason of
 * at most msg_len bytes. */
psatd_status psatd_plan_validate(const psatd_plan_desc* desc, char* msg, size_t msg_len);

/* Host-only: compute the guard-exchange copy blocks of a valid description.
 * Writes up to `cap` blocks to `out` (may be NULL when cap = 0) and the total
 * count to *count. */
psatd_status psatd_exchange_blocks(const psatd_plan_desc* desc, psatd_copy_block* out,
                                   int64_t cap, int64_t* count);

/* Host-only: where the deferred guard exchange (see PSATD_EAGER_EXCHANGE)
 * makes the forward pass read plane z of box `box` (paper Fig. 1, step (ii)
 * folded into the next step).  For every cell (y, x) of the padded plane, at
 * index y * n[0] + x of the caller's arrays of n[0] * n[1] entries:
 * src_box / src_cell = the box and the linear cell index (x fastest, then y,
 * then z) of the cell whose value is read there -- the owning interior cell
 * for a guard cell that has an owner, the cell itself otherwise.  *is_grid = 1
 * when the plane is the 3 x 3 rectangle grid the kernels use (the indices are
 * then produced from that grid form), 0 when only the rectangle list applies.
 * Errors: PSATD_ERR_INVALID_ARG for an invalid description, box or plane, or
 * a NULL output. */
psatd_status psatd_plane_gather(const psatd_plan_desc* desc, int32_t box, int32_t z,
                                int32_t* src_box, int64_t* src_cell, int32_t* is_grid);

/* Build a plan: validate, build the copy blocks and work lists, allocate the
 * spectral workspace and tables, and generate the FP64 tables (twiddles,
 * modified wavenumbers k_p, Yee phase factors, PSATD coefficients) with
 * device kernels on `stream`.  Returns when the plan is ready.  On error
 * *out is set to NULL and nothing is leaked. */
psatd_status psatd_plan_create(const psatd_plan_desc* desc, void* stream, psatd_plan** out);

/* Free every resource of the plan (synchronises the device first). NULL is ok. */
psatd_status psatd_plan_destroy(psatd_plan* plan);

/* Element offset and element count of box `box` inside every field buffer. */
psatd_status psatd_plan_layout(const psatd_plan* plan, int32_t box, int64_t* elem_offset,
                               int64_t* elems);

/* Bytes of one field-component buffer (all boxes) and of the plan-owned
 * device memory (spectral workspace plus tables). */
psatd_status psatd_plan_memory(const psatd_plan* plan, size_t* field_bytes,
                               size_t* workspace_bytes);

/* S4 (and the initial fill, S0): copy every guard cell of E, B from its
 * owning interior cell; with `src` non-NULL also J and rho.  Asynchronous. */
psatd_status psatd_guard_exchange(psatd_plan* plan, const psatd_fields* fields,
                                  const psatd_sources* src, void* stream);

/* Advance `nsteps` >= 0 steps of S1..S4 in place on `fields` (and rho).
 * Guards of E, B must be consistent on entry (psatd_guard_exchange) and are
 * consistent on return; between the steps of one call they may stay stale
 * in memory (PSATD_EAGER_EXCHANGE).  Asynchronous on `stream`. */
psatd_status psatd_push(psatd_plan* plan, const psatd_fields* fields,
                        const psatd_sources* src, int32_t nsteps, void* stream);

/* psatd_push for fields in HOST memory (no counterpart in the paper: the
 * host path of a caller whose fields live on the CPU).  in / out: six host
 * component buffers each (same layout as the device buffers, field_bytes
 * each; they may be the same buffers; page-locked memory copies fastest).
 * The fields are copied to plan-owned device staging buffers (allocated by
 * the first call, 6 x field_bytes, kept until psatd_plan_destroy; that first
 * call therefore allocates and should come before any stream capture), by
 * the copy engines or by a copy kernel through the buffers' device mapping
 * (PSATD_TUNE_HOST_COPY); then `nsteps` steps run as in psatd_push (`src`:
 * device sources as there), and the results are copied back the same way.
 * The copies run component by component on a plan-owned side stream; for
 * the vacuum form the first step's forward x, y transforms and the last
 * step's inverse y, x transforms also go component by component, so that
 * the copy of one component overlaps the transforms of its neighbour (the
 * same kernels on the same data: the results equal psatd_push's bit for
 * bit).  Asynchronous on `stream`: the host buffers must stay valid, and `in`
 * unchanged, until `stream` has passed this call; work queued on `stream`
 * afterwards sees the results in `out`.  Errors as psatd_push. */
psatd_status psatd_push_host(psatd_plan* plan, const psatd_fields* in, const psatd_fields* out,
                             const psatd_sources* src, int32_t nsteps, void* stream);

/* psatd_push for fields held on the host as whole-domain arrays (no
 * counterpart in the paper: the host path of a caller who stores the global
 * fields, not the padded boxes).  in / out: six host arrays each of
 * global_n[0] * global_n[1] * global_n[2] elements (x fastest, then y, z;
 * the plan's precision; in and out may be the same).  The domain is copied
 * to the device (as in psatd_push_host), scattered into the plan's padded
 * boxes, guards included (the dual-grid coupling of the plan with one box
 * covering the domain), pushed `nsteps` steps, and the box interiors are
 * gathered back and copied to `out`, component by component as in
 * psatd_push_host (the copy of one component also overlaps the scatter or
 * the gather of its neighbour).  The first call allocates plan-owned
 * device buffers (6 x the domain and 6 x field_bytes) and the coupling, kept
 * until psatd_plan_destroy; make it before any stream capture.  Not for
 * PSATD_DECOMP_INDEPENDENT (PSATD_ERR_STATE).  Asynchronous on `stream`, with
 * the same rules for the host buffers as psatd_push_host. */
psatd_status psatd_push_host_global(psatd_plan* plan, const psatd_fields* in, const psatd_fields* out,
                                    const psatd_sources* src, int32_t nsteps, void* stream);

/* S1 alone for one component: unnormalised 3D R2C FFT of every box of
 * `field` (device, one component buffer) into `spectrum` (device, complex
 * float2/double2, box b at psatd_plan_spectrum_layout offset, element
 * (mx, my, mz) at mx + (n[0]/2+1)*(my + n[1]*mz)). */
psatd_status psatd_forward_fft(psatd_plan* plan, const void* field, void* spectrum,
                               void* stream);

/* S3 alone: C2R inverse (with the 1/(n0 n1 n2) factor) of `spectrum` into
 * every cell of `field`.  `spectrum` is used as scratch and overwritten. */
psatd_status psatd_inverse_fft(psatd_plan* plan, void* spectrum, void* field, void* stream);

/* Complex-element offset and count of box `box` in a spectrum buffer. */
psatd_status psatd_plan_spectrum_layout(const psatd_plan* plan, int32_t box,
                                        int64_t* elem_offset, int64_t* elems);

/* ---- One group spread over several ranks (paper Sec. 2.4.1: the group's
 * FFT distributed over the MPI ranks of a sub-communicator, axis by axis with
 * a transposition before each axis whose lines are split; Sec. 2.6: the
 * "optimized communication strategy" keeps the spectrum in the transposed
 * layout, solves Maxwell's equations there and starts the inverse transform
 * from it, so a step moves the spectrum twice instead of four times).
 *
 * A plan of one box -- the group, periodic along y and z inside its FFT (no
 * guards on the y and z faces) -- becomes rank `rank` of `world` ranks that
 * share the group's FFT.  Real space is split in z slabs: the rank holds the
 * planes [z0, z1) of the box (every y and x, x-face guards included).  After
 * the x and y transforms, one all-to-all gives every rank the spectrum rows
 * my in [y0, y1) for every z; the rank transforms z, updates every mode (the
 * wavenumbers from the global indices) and transforms z back in that layout,
 * and a second all-to-all returns the rows to the slabs for the inverse y and
 * x transforms.  The library does the rank's device work; the caller moves
 * the spectrum (NCCL, MPI, or copies): rank r sends the rows [y0_s, y1_s) of
 * every plane of its slab to rank s, which stores them at z planes [z0_r,
 * z1_r) of its rows buffer, and back.  Slabs and rows are split as evenly as
 * possible, the larger parts first (the first n % world ranks have one more
 * plane or row).  The device work runs on the generic kernels, in the plan's
 * precision and form; a constant current is transformed every step.
 *
 * Buffers (caller-owned, device, 16-byte aligned, components contiguous):
 *   slab fields (psatd_fields / psatd_sources as in psatd_push): per
 *     component (z1 - z0) * n1 * n0 reals, x fastest;
 *   slab spectrum: F components, each (z1 - z0) * n1 * (n0/2 + 1) complex in
 *     the order (z, y, mx), component c at c * (z1 - z0) * n1 * (n0/2 + 1);
 *   rows spectrum: F components, each n2 * (y1 - y0) * (n0/2 + 1) complex in
 *     the order (z, y, mx);
 *   F = 6 (vacuum), 9 (E, B, J), 10 (E, B, rho, J) slots in the order of the
 *   fields and sources (psatd_dist_forward_xy writes all F; psatd_dist_z_update
 *   reads F and writes E, B (and rho'); psatd_dist_inverse_yx reads those).
 *
 * psatd_plan_distribute: PSATD_ERR_INVALID_ARG for a plan of several boxes,
 * y or z guards, absorbing layers, or rank/world outside 0 <= rank < world <=
 * min(n1, n2); PSATD_ERR_STATE when the plan is already distributed.  Builds
 * the rank's job lists (plan-owned device memory).  The other calls return
 * PSATD_ERR_STATE before it, and are asynchronous on `stream`. */
psatd_status psatd_plan_distribute(psatd_plan* plan, int32_t world, int32_t rank);
/* The rank's slab [z0, z1) and spectrum rows [y0, y1) (any pointer may be NULL). */
psatd_status psatd_dist_bounds(const psatd_plan* plan, int32_t* z0, int32_t* z1, int32_t* y0, int32_t* y1);
/* S1 (x, y): R2C along x and FFT along y of every slot of the slab. */
psatd_status psatd_dist_forward_xy(psatd_plan* plan, const psatd_fields* slab, const psatd_sources* sources,
                                   void* slab_spectrum, void* stream);
/* S1 (z), S2, S3 (z) on the rank's rows, in place. */
psatd_status psatd_dist_z_update(psatd_plan* plan, void* rows_spectrum, void* stream);
/* S3 (y, x): inverse y FFT and C2R along x (the group's 1/(n0 n1 n2)) of the
 * output slots into the slab's interior x cells (x-face guards untouched);
 * `slab_spectrum` is overwritten. */
psatd_status psatd_dist_inverse_yx(psatd_plan* plan, void* slab_spectrum, const psatd_fields* slab,
                                   const psatd_sources* sources, void* stream);

/* Wait for the plan's last stream and return the first pending error
 * (CUDA error or device-side status word). */
psatd_status psatd_sync_status(psatd_plan* plan);

/* Static text for a status code. */
const char* psatd_status_string(psatd_status s);

/* Text of the last error of `plan`, or of the calling thread's last failed
 * psatd_plan_create / psatd_plan_validate when plan is NULL.  Never NULL. */
const char* psatd_last_error(const psatd_plan* plan);

/* ---- Dual-grid coupling (paper Sec. 2.5.2, "dual grid decomposition") ------
 * A second decomposition G1 of the plan's global domain -- e.g. the grid of the
 * particle and particle-mesh operations of a PIC code, with its own sub-domain
 * boundaries and thin guard layers -- coupled to the plan's FFT boxes G2.
 * Every cell of every destination box (guards included) takes the value of the
 * source grid's interior cell with the same global index (periodic axes wrap;
 * non-periodic axes give 0 outside the domain):
 *   PSATD_G1_TO_G2  fills the FFT boxes, guards included, before a push (the
 *                   guard exchange of the FFT grid is then already done);
 *   PSATD_G2_TO_G1  copies the pushed fields back (the FFT grid's guard cells
 *                   are not read; G1's guards get their owners' new values).
 * G1 boxes use psatd_box: n counts cells including guards (any size >= 1, no
 * FFT constraint), origin is the global index of the first interior cell; the
 * interiors must tile the domain exactly.  Not for PSATD_DECOMP_INDEPENDENT. */
typedef struct psatd_coupling psatd_coupling;
#define PSATD_G1_TO_G2 0
#define PSATD_G2_TO_G1 1

/* Host-only: the copy blocks of one direction (src_box indexes the source
 * grid, dst_box the destination grid; src_box = -1: zero fill).  Same output
 * convention as psatd_exchange_blocks. */
psatd_status psatd_coupling_blocks(const psatd_plan_desc* g2, int32_t num_g1_boxes, const psatd_box* g1_boxes,
                                   int32_t direction, psatd_copy_block* out, int64_t cap, int64_t* count);

/* Build the coupling of `plan` (G2) with the G1 boxes: validates them,
 * computes both directions' copy blocks and uploads them (plan's device).
 * The coupling borrows the plan: destroy it before the plan. */
psatd_status psatd_coupling_create(psatd_plan* plan, int32_t num_g1_boxes, const psatd_box* g1_boxes,
                                   psatd_coupling** out);
psatd_status psatd_coupling_destroy(psatd_coupling* coupling);

/* Element offset and count of G1 box `box` in a G1 component buffer (boxes
 * concatenated at 64-element-aligned offsets, x fastest, precision of the
 * plan). */
psatd_status psatd_coupling_layout(const psatd_coupling* coupling, int32_t box, int64_t* elem_offset,
                                   int64_t* elems);

/* Copy `nfields` component buffers (device pointers, 16-byte aligned, same
 * component order on both grids) in `direction` on `stream`, asynchronously:
 * one batched copy kernel.  Source and destination buffers must not overlap. */
psatd_status psatd_couple(psatd_coupling* coupling, int32_t direction, void* const* g1_fields,
                          void* const* g2_fields, int32_t nfields, void* stream);

/* Device pointer of stored split part q (0..5: E_xy, E_yz, E_zx, B_xy, B_yz,
 * B_zx) of a plan with absorbing layers: one plan-owned buffer with the
 * layout of a field buffer (interior cells meaningful), read and written by
 * every psatd_push.  PSATD_ERR_STATE for a plan without layers. */
psatd_status psatd_plan_pml_part(const psatd_plan* plan, int32_t q, void** part);

/* Number of kernel launches issued by the last push call (psatd_push, or
 * psatd_push_host_global with its copy kernels, scatters and gathers; host
 * count). */
int64_t psatd_last_launch_count(const psatd_plan* plan);

/* Number of boxes that run on the fast plane kernels (all three FFT lengths
 * have a two-pass register schedule and the planes fit in shared memory);
 * -1 for a NULL plan. */
int32_t psatd_plan_fast_boxes(const psatd_plan* plan);

/* Number of boxes that run on the pencil kernels (two-pass lengths up to 512
 * along x and y, up to 256 along z in FP32 / 128 in FP64, planes too large
 * for the plane kernels); the remaining boxes run on the generic multi-pass
 * kernels.  -1 for a NULL plan.  No counterpart in the paper (a property of
 * this implementation's kernel selection). */
int32_t psatd_plan_pencil_boxes(const psatd_plan* plan);

/* 1 when the plan defers each step's guard exchange into the next step's
 * forward pass (see PSATD_EAGER_EXCHANGE), 0 when every step stores its
 * guards, -1 for a NULL plan. */
int32_t psatd_plan_deferred_exchange(const psatd_plan* plan);

/* ---- Tuning knobs (no counterpart in the paper: launch parameters of this
 * implementation's kernels, chosen per plan by measurement -- see the
 * autotuner of the Python package).  Results do not depend on any knob.
 * Every knob can be given at plan creation (psatd_plan_desc.tuning); the
 * ones marked "runtime" can also be changed later with psatd_plan_tune,
 * which drops the plan's captured CUDA graphs.
 *   PSATD_TUNE_Z_PREFETCH    (runtime) register z kernel (the fused z FFT +
 *                            update pass): every CTA first prefetches into L2
 *                            the input tile of the CTA launched `value` blocks
 *                            after it (0 = off; 0 <= value <= 2^20;
 *                            default 64).
 *   PSATD_TUNE_PENCIL_ROWS_KB  pencil x-pass batching: shared memory (KiB)
 *                            for the rows one CTA transforms (8 .. 200;
 *                            default 64).
 *   PSATD_TUNE_Z_TILE        mx columns per tile of the shared-memory plane
 *                            family's and the pencil family's z pass (1 ..
 *                            8 in FP32, 1 .. 4 in FP64; default the maximum).
 *   PSATD_TUNE_HOST_COPY     (runtime) psatd_push_host's copies: 1 (default)
 *                            = a copy kernel on the SMs reading and writing
 *                            the host buffers through their device mapping
 *                            when every buffer is page-locked, mapped and
 *                            16-byte aligned (else the copy engines); 0 = the
 *                            copy engines, one stream per component.
 *   PSATD_TUNE_PENCIL_REG_Z  FP32 boxes whose z length has a register z
 *                            kernel (48, 60, 80, 96, 120), on the pencil
 *                            kernels, or on the plane kernels in a batch of
 *                            several z lengths: 1 (default) = that kernel
 *                            does their z pass, 0 = the shared-memory z
 *                            kernel of their family.
 *   PSATD_TUNE_Z_ONE_LAUNCH  (runtime) those boxes' z pass: 0 (default) = one
 *                            launch per z length, 1 = one persistent launch
 *                            for every z length (2 CTAs per SM, each taking
 *                            every grid-th tile in turn and prefetching its
 *                            next tile into L2).
 *   PSATD_TUNE_REG_PLANES    FP32 boxes whose plane shape (n0/2, n1) has
 *                            register plane kernels (n0/2 in 24, 30, 40, 48,
 *                            60; n1 in 48, 60, 80, 96, 120): 1 (default) =
 *                            those kernels (one launch per shape), 0 = the
 *                            family the box would take without them (pencil,
 *                            or the shared-memory plane kernels with
 *                            PSATD_PLANE_KERNELS).
 * psatd_plan_create and psatd_plan_validate return PSATD_ERR_INVALID_ARG for
 * an unknown knob or a value out of range, psatd_plan_tune also for a knob
 * that is not runtime; psatd_plan_tuning returns the knob's value, or -1 for
 * an unknown knob, a NULL plan, or a plan whose kernels do not use the knob. */
#define PSATD_TUNE_Z_PREFETCH 1
#define PSATD_TUNE_PENCIL_ROWS_KB 2
#define PSATD_TUNE_Z_TILE 3
#define PSATD_TUNE_HOST_COPY 4
#define PSATD_TUNE_PENCIL_REG_Z 5
#define PSATD_TUNE_Z_ONE_LAUNCH 6
#define PSATD_TUNE_REG_PLANES 7
psatd_status psatd_plan_tune(psatd_plan* plan, int32_t knob, int32_t value);
int32_t psatd_plan_tuning(const psatd_plan* plan, int32_t knob);

/* Kernel kinds reported by psatd_plan_kernel_times. */
#define PSATD_KERNEL_KINDS 6 /* 0 fwd_x, 1 col forward, 2 z_update, 3 col inverse, 4 inv_x, 5 exchange */

/* Diagnostics: with enable != 0, psatd_push brackets every kernel launch with
 * CUDA events recorded on its stream (no extra synchronisation). */
psatd_status psatd_plan_set_timing(psatd_plan* plan, int32_t enable);

/* Synchronise the plan's last stream, then add the device time (ms) and the
 * number of launches of every kernel kind recorded since the previous call
 * into ms[0..n) and launches[0..n) (n <= PSATD_KERNEL_KINDS; either array may
 * be NULL), and forget the records. */
psatd_status psatd_plan_kernel_times(psatd_plan* plan, double* ms, int64_t* launches, int32_t n);

/* ---------------------------------------------------------------------------
 * Push without device allocation (the paper has no counterpart: this is a
 * service for callers that may not allocate device memory, e.g. code running
 * under a host framework that owns every device allocation, or a fixed-memory
 * real-time loop).
 *
 * Advances one periodic box of n[0] x n[1] x n[2] cells (no guards, the
 * 'global' decomposition), FP32, vacuum, by `nsteps` steps of S1..S3, in place
 * on the caller's six FP32 device buffers (x fastest, 16-byte aligned, each
 * n[0]*n[1]*n[2] floats).  order_p, dx, dt, c as in psatd_plan_desc
 * (eps0 is irrelevant in vacuum).  The result equals psatd_push on a
 * one-box PSATD_DECOMP_GLOBAL FP32 vacuum plan.
 *
 * Nothing is allocated: the spectral workspace, tables and work lists live in
 * one static device array of PSATD_STATIC_SCRATCH_BYTES (64 MiB), reserved on
 * every GPU that loads the library until the process exits.  A box whose
 * needs exceed it (a 128^3 box fits, 144^3 does not) is rejected with
 * PSATD_ERR_UNSUPPORTED_SIZE and a message giving both byte counts.  All calls
 * on a device share the array; calls that overlap on the GPU race and give
 * wrong results.  The first call on each device looks up the array's address
 * and sets kernel attributes: make it before any stream capture.  Errors are
 * reported through psatd_last_error(NULL).
 * ------------------------------------------------------------------------- */
#define PSATD_STATIC_SCRATCH_BYTES (64ull << 20)

psatd_status psatd_push_box_static(const int32_t n[3], int32_t order_p, const double dx[3],
                                   double dt, double c, const psatd_fields* fields,
                                   int32_t nsteps, void* stream);

#ifdef __cplusplus
}
#endif

#endif /* PSATD_H */
