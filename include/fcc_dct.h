/*
 * fcc_dct.h -- C ABI of libfccdct, a CUDA (sm_103a) implementation of the FCC
 * cosine transform DCT_{n x n x n} of Seifert, Hueper and Uhl, "Fast cosine
 * transform for FCC lattices" (2018).
 *
 * The operation (Def. 2 and its explicit matrix form, Sec. 4.A):
 *
 *   y[i,l,q] = sum_{0 <= j,k,p < n} x[j,k,p] * T_{j,k,p}(theta_{i,l,q}),
 *   theta_{i,l,q} = ((1/8 + i)/n, l/n, (3/8 + q)/n)          (Lemma 1),
 *   T_k(theta)    = (1/24) sum_{w in W} exp(2 pi i (w k).theta)
 *                   (Def. 1 with the power form of Sec. 3; W is the group
 *                   of order 24 generated by the printed s1, s2, s3, acting
 *                   on k from the left).
 *
 * "forward" is y = D x (coefficients of the basis b_n -> values at the n^3
 * common zeros), "inverse" is x = D^{-1} y (the inverse of the CRT
 * isomorphism of Lemma 2, which exists because the zeros are distinct) and
 * "adjoint" is D^H g.  No normalisation beyond the 1/24 inside T_k.
 *
 * Layouts.  A volume is n^3 values, index (a,b,c) at a*n*n + b*n + c (last
 * index fastest).  Coefficient volumes are indexed (j,k,p), point volumes
 * (i,l,q).  A batch is `batch` volumes back to back.  Complex values are
 * interleaved (re, im) pairs of the dtype's real type.
 *
 *   dtype          forward in      forward out     inverse/adjoint in/out
 *   FCC_R64        double          complex double  complex double -> double
 *   FCC_C64        complex double  complex double  complex double -> complex
 *   FCC_R32        float           complex float   complex float  -> float
 *   FCC_C32        complex float   complex float   complex float  -> complex
 *   FCC_R32_*X3    as FCC_R32
 *
 * For the real dtypes the inverse returns the real part of D^{-1} y (exact
 * when y = D x for a real x) and the adjoint returns Re(D^H g), the adjoint
 * of the real-linear map x -> D x.
 *
 * Ownership and execution.  `in` and `out` are DEVICE pointers owned by the
 * caller, 16-byte aligned, not overlapping.  Calls are asynchronous on
 * `stream` (a cudaStream_t passed as void*; NULL = legacy default stream)
 * and never synchronise the host.  A plan owns its device tables and
 * workspace; it is not thread safe: use one plan from one host thread and
 * one stream at a time.  All entry points return a status code; no C++
 * exception crosses the ABI.
 */
#ifndef FCC_DCT_H
#define FCC_DCT_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct fcc_plan fcc_plan;

typedef enum {
    FCC_OK = 0,
    FCC_ERR_INVALID_ARG = 1, /* NULL, misaligned or overlapping buffers, bad order/batch/dtype */
    FCC_ERR_UNSUPPORTED = 2, /* valid request this build does not implement */
    FCC_ERR_ALLOC = 3,       /* host or device allocation failed; nothing leaked */
    FCC_ERR_CUDA = 4,        /* a CUDA runtime call or kernel launch failed */
    FCC_ERR_TIMEOUT = 5      /* a device-side wait exceeded its bound */
} fcc_status;

typedef enum {
    FCC_R64 = 0,
    FCC_C64 = 1,
    FCC_R32 = 2,
    FCC_C32 = 3,
    FCC_R32_TF32X3 = 4,   /* FP32 storage; the forward orbit cores on the tensor cores (TF32, 3-term inputs) */
    FCC_R32_BF16X3 = 5,   /* FP32 storage; the forward orbit cores on the tensor cores (BF16, 3-term inputs) */
    FCC_R32_BF16X6 = 6    /* 3-way split of both operands, 6 products: the core's low parts are exactly
                             zero, so this runs the 3 products of FCC_R32_BF16X3 (identical results) */
} fcc_dtype;

/* Largest supported order n. */
#define FCC_MAX_ORDER 512

/*
 * Build a plan for `batch` volumes of order `order` (1 <= order <=
 * FCC_MAX_ORDER, batch >= 1) in `dtype`.  Does the host-side set-up (the
 * orbit partition of Z_n^3 under W and its class cores, Sec. 3 / Def. 2),
 * allocates and fills device tables on the current device.  Returns NULL
 * on error; fcc_dct_last_error() tells why.
 */
fcc_plan* fcc_dct_plan(int order, int batch, int dtype);

/*
 * Rendering of voxel data as lattice cells (Sec. 5, Fig. 4; the paper shows
 * figures only, this is a headless restatement): every data point of an n^3
 * volume (device, FP32, [n][n][n], the layout of a real forward input) is
 * drawn as the cell around its lattice point -- FCC_CELL_CUBE: the unit cube
 * around (i, l, q) on the cubic lattice (Fig. 4a); FCC_CELL_RHOMBIC_DODECAHEDRON:
 * the Voronoi cell of z = (i + q, i + l, l + q) in the FCC lattice
 * D3 = {z in Z^3 : z1 + z2 + z3 even} (Fig. 4b) -- with the data value as
 * opacity (clamped to [0, 1]; 0 invisible, 1 opaque).  An orthographic ray
 * marcher looks at the centre of the cells' bounding box from the direction
 * (cos e cos a, cos e sin a, sin e) (a = azimuth, e = elevation, radians),
 * the width x height image spanning the box's bounding sphere; along each ray
 * a sample every `step` (lattice units) inside a cell of value v has opacity
 * 1 - exp(-kappa v step) and emits v, composited front to back.  Writes the
 * grey level of every pixel to image[height][width] (device, FP32),
 * asynchronously on `stream`.  FCC_ERR_INVALID_ARG for NULL pointers, n outside
 * 1..FCC_MAX_ORDER, an unknown cell kind, sizes outside 1..16384, kappa or
 * step not positive, or more than 10^6 steps per ray.
 */
typedef enum { FCC_CELL_CUBE = 0, FCC_CELL_RHOMBIC_DODECAHEDRON = 1 } fcc_cell;
fcc_status fcc_render_cells(const float* volume, int n, int cells, float azimuth, float elevation, float kappa,
                            float step, int width, int height, float* image, void* stream);

/*
 * The paper's own fast algorithm (Sec. 4.B, eq. FastAlgorithm): the radix-2x2x2
 * factorisation
 *   DCT_n(c) = P_n . (sum over i in {0,1}^3 of DCT_m((c + i)/2)) . (DCT_2(c) (x) 1_{m^3}) . B_n(c),
 * n = 2m, evaluated recursively on the GPU down to the 8 x 8 DCT_2 of Def. 2.
 * The basis change B_n, which the paper leaves to future work, is derived from
 * its definition at plan time: B_n^{-1} column (efg, abc) is T_{abc} T_{m(e,f,g)}
 * expanded with the mother recurrence (Prop. 1 (iv)) and reduced with the
 * ideal T_{n e_j} = T_{e_j}(c) (Lemma 2), assembled in FP64 on the host and
 * inverted on the GPU.  A second, independent evaluation of the transform
 * (not the fast path: its FP32 error grows about tenfold per level, and B_n is
 * dense-stored).  order: 2, 4, 8 or 16; dtype: FCC_C64 (FP64) or FCC_C32 (FP32
 * arithmetic throughout, to measure how the recursion rounds); v, d: the shift
 * c = v / d (v = NULL: (1/8, 0, 3/8)).  The plan serves fcc_dct_forward only
 * (complex coefficients in, complex point values out, the layouts of the
 * other plans); every other call on it returns FCC_ERR_UNSUPPORTED.  Plan
 * creation synchronises the device and takes up to a few seconds at order 16
 * (B_16 is 4096 x 4096).  NULL on error: FCC_ERR_INVALID_ARG, FCC_ERR_ALLOC,
 * FCC_ERR_UNSUPPORTED (a singular B_n^{-1}).
 */
fcc_plan* fcc_dct_plan_radix2(int order, int batch, int dtype, const int* v, int d);

/*
 * Statistics of a radix-2 plan: level = k (k = order, order/2, ... >= 4):
 * non-zeros per row of B_k (entries above 1e-12 of the largest, averaged over
 * the level's shifts) and its largest |entry|, returns the number of shifts at
 * that level; level = 0: complex multiply-adds per point of one transform
 * (the non-zeros of every B_k, 64 per column block of DCT_2 (x) 1, 64 per
 * DCT_2), returns 0.  -1 (FCC_ERR_INVALID_ARG) for other plans or levels.
 */
int fcc_dct_radix2_stats(const fcc_plan* plan, int level, double* nnz_per_row, double* max_abs, double* macs_per_point);

/*
 * Plan for a ragged batch: `count` volumes whose orders are orders[0..count)
 * stored back to back (volume v starts at sum_{u<v} orders[u]^3 values).
 * Same layouts and dtypes as fcc_dct_plan.  `orders` is a host array read
 * during the call only.
 */
fcc_plan* fcc_dct_plan_ragged(const int* orders, int count, int dtype);

/*
 * Plan for the skew transform DCT_{n x n x n}(r,s,t) of Def. 2 (its explicit
 * matrix form, Sec. 4.A; the points are the common zeros of Lemma 2):
 *
 *   y[i,l,q] = sum_{j,k,p} x[j,k,p] T_{j,k,p}(((r+i)/n, (s+l)/n, (t+q)/n)),
 *   (r, s, t) = (v[0], v[1], v[2]) / d,
 *
 * with 1 <= d <= FCC_MAX_SHIFT_DEN and |v[i]| <= FCC_MAX_SHIFT_NUM (`v` is a
 * host array of 3 ints read during the call only).  (1/8, 0, 3/8), in any
 * form such as (2, 0, 6) / 16, is the plan of fcc_dct_plan.  Same layouts,
 * entry points and errors otherwise, with these differences for any other
 * shift:
 *   - dtypes FCC_R64, FCC_C64, FCC_R32, FCC_C32 only (the tensor-core dtypes
 *     return NULL with FCC_ERR_UNSUPPORTED: their exact core split needs the
 *     8th-root cores of the shift (1/8, 0, 3/8));
 *   - D is invertible only when every W-orbit block is; this holds for the
 *     shifts (c + a)/2 (a in {0,1}^3) of the radix-2 step of Sec. 4.B, c =
 *     (1/8, 0, 3/8), and fails for most others (e.g. (0,0,0), (1,1,1)/4).
 *     For a singular D the plan is still built (forward and adjoint work)
 *     and fcc_dct_inverse / fcc_dct_inverse_host return FCC_ERR_UNSUPPORTED;
 *   - fcc_dct_inverse_static returns FCC_ERR_UNSUPPORTED.
 */
#define FCC_MAX_SHIFT_DEN 1024
#define FCC_MAX_SHIFT_NUM 65536
fcc_plan* fcc_dct_plan_skew(int order, int batch, int dtype, const int* v, int d);

/* y = D x over the plan's batch; in: coefficients, out: point values. */
fcc_status fcc_dct_forward(fcc_plan* plan, const void* in, void* out, void* stream);

/* x = D^{-1} y; in: point values (complex), out: coefficients. */
fcc_status fcc_dct_inverse(fcc_plan* plan, const void* in, void* out, void* stream);

/* x = D^H g (real dtypes: Re D^H g); in: point values (complex). */
fcc_status fcc_dct_adjoint(fcc_plan* plan, const void* in, void* out, void* stream);

/*
 * End-to-end forms taking HOST buffers: copy `host_in` to plan-owned device
 * memory, transform, copy the result to `host_out`, all ordered after the
 * work already on `stream`.  The caller synchronises `stream` before reading
 * host_out.  Pinned (page-locked) host buffers make the copies asynchronous;
 * for uniform plans of 4 or more volumes the copies of ~32 MB chunks of
 * volumes run on two plan-owned streams, overlapping the transform of the
 * neighbouring chunks (results are identical to the device-pointer calls).
 */
fcc_status fcc_dct_forward_host(fcc_plan* plan, const void* host_in, void* host_out, void* stream);
fcc_status fcc_dct_inverse_host(fcc_plan* plan, const void* host_in, void* host_out, void* stream);

/*
 * Hermitian-packed forward and inverse of real plans (FCC_R64, FCC_R32 and
 * the tensor-core dtypes) at the canonical shift (1/8, 0, 3/8).
 *
 * For real x the rows of the explicit matrix of Def. 2 come in conjugate
 * pairs: y[pi(i,l,q)] = conj(y[i,l,q]) with the involution
 * pi(i,l,q) = ((i - l) mod n, (-l) mod n, (q - l) mod n), whose fixed points
 * (row l = 0) carry real values.  So the n^3 complex values y = D x of a real
 * volume are fixed by n^3 reals.  The packed volume (n^3 reals of the
 * dtype's real type, point order (i,l,q)) holds at point a = (i,l,q)
 *     Re y[a]    if 2l < n, or 2l = n and 2q < n   ("primary" points),
 *     -Im y[a]   otherwise (= Im y at the primary partner pi(a)).
 * Unpacking: y[a] = pk[a] + i pk[pi(a)] at a primary point (pk[a] when
 * l = 0), y[a] = pk[pi(a)] - i pk[a] elsewhere.
 *
 * fcc_dct_forward_packed: in = coefficients (real), out = packed D x.
 * fcc_dct_inverse_packed: in = a packed volume (it stands for a y with the
 * conjugate symmetry above), out = D^{-1} y (real coefficients; exact
 * inverse of the packed forward).  Both move half the bytes of the complex
 * form's point values.  Buffers: points * sizeof(real) bytes each, device
 * pointers, 16-byte aligned, not overlapping.  Errors: FCC_ERR_UNSUPPORTED
 * for complex dtypes, skew plans and (inverse) singular plans;
 * FCC_ERR_INVALID_ARG as for fcc_dct_forward; FCC_ERR_ALLOC when the first
 * call cannot allocate its workspace (two chunks of complex intermediate per
 * internal stream, held by the plan).  The *_host forms take host buffers as
 * fcc_dct_forward_host does.
 */
fcc_status fcc_dct_forward_packed(fcc_plan* plan, const void* in, void* out, void* stream);
fcc_status fcc_dct_inverse_packed(fcc_plan* plan, const void* in, void* out, void* stream);
fcc_status fcc_dct_forward_packed_host(fcc_plan* plan, const void* host_in, void* host_out, void* stream);
fcc_status fcc_dct_inverse_packed_host(fcc_plan* plan, const void* host_in, void* host_out, void* stream);

/* Number of volumes, total points (sum of n^3) and element counts of the
 * forward input / output, for sizing buffers. */
int fcc_dct_batch(const fcc_plan* plan);
int64_t fcc_dct_points(const fcc_plan* plan);
/* Bytes of the forward input and output of the whole batch. */
int64_t fcc_dct_in_bytes(const fcc_plan* plan);
int64_t fcc_dct_out_bytes(const fcc_plan* plan);

/* Kernel launches one forward / inverse call enqueues (for reporting). */
int fcc_dct_launches(const fcc_plan* plan, int which /* 0 fwd, 1 inv, 2 adj, 3 fwd packed, 4 inv packed */);

/*
 * Tracing: every entry-point call and every kernel launch it makes open an
 * NVTX range (host side; named after the call, e.g. "fcc_dct_forward", and
 * after the kernel kind, e.g. "mix_tc_fwd", "fft_slab"), for timeline tools.
 * Without a tool attached the ranges cost a function-pointer check.
 *
 * Optional per-kernel timing.  When enabled, every kernel launch the plan
 * enqueues is bracketed by a pair of CUDA events on the launch stream.
 * fcc_dct_profile_read() waits for the recorded events, then writes for up
 * to `cap` kernel kinds their name (NUL-terminated, 48 bytes each, into
 * names[48*i]), summed duration in milliseconds and launch count, clears
 * the record and returns the number of kinds (or -1 on error).
 */
fcc_status fcc_dct_profile_enable(fcc_plan* plan, int enable);
int fcc_dct_profile_read(fcc_plan* plan, char* names, double* ms, int* launches, int cap);

/*
 * Measurement aid (no counterpart in the paper): replays the global-memory
 * accesses of the forward tensor-core orbit mixing -- the gathers of all 24
 * slots of both volumes of every pair and the stores of the canonical slots,
 * at the addresses, in the chunks and in the launch geometry (grid, block,
 * shared memory, so the same blocks per SM) of fcc_dct_forward's mixing
 * stage -- with no arithmetic, on `stream` alone.  Its time is the ceiling
 * that the mixing's access pattern puts on the mixing kernel (the launches
 * appear as "mix_replay" in the per-kernel timing).  in: the forward's input
 * (real volumes, device, 16-byte aligned); out: a buffer of the forward's
 * output size that receives meaningless values (not overlapping in).
 * Uniform real tensor-core plans at the canonical shift with batch >= 2 and
 * free orbits; FCC_ERR_UNSUPPORTED otherwise, FCC_ERR_INVALID_ARG for null,
 * misaligned or overlapping buffers.
 */
fcc_status fcc_dct_diag_mixing_replay(fcc_plan* plan, const void* in, void* out, void* stream);

/*
 * Inverse transform that allocates nothing (the paper has no counterpart).
 *
 * Some callers cannot allocate device memory at the moment they need the
 * inverse: code running inside an allocator or memory-pool callback, or a
 * latency-critical loop in which a cudaMalloc would synchronise the device
 * with work already running.  This entry point computes exactly what
 * fcc_dct_inverse computes, but its complex workspace lives in one
 * file-scope device array of FCC_STATIC_SCRATCH_BYTES that every GPU which
 * loads the library holds until the process exits; it calls no cudaMalloc,
 * cudaFree or other allocating routine.  The plan (created earlier, when
 * allocation was allowed) supplies the read-only tables; `in` and `out` are
 * the caller's device buffers as for fcc_dct_inverse.
 *
 * Limits: FP32 plans only (FCC_R32, FCC_C32) whose largest volume fits the
 * array as complex values (n^3 * 8 bytes <= FCC_STATIC_SCRATCH_BYTES, i.e.
 * n <= 128); anything else returns FCC_ERR_UNSUPPORTED without launching.
 * Volumes are processed one chunk at a time on `stream` only.
 *
 * Set-up: the first call on each device looks up the array's device address
 * (cudaGetSymbolAddress) with that device current; make that first call
 * before any stream capture.  The array is shared by all calls and keeps
 * the last call's contents; nothing in it needs to start at zero (every
 * value is written before it is read).  Calls whose work overlaps on the GPU
 * (different streams, or different host threads) race on the array and
 * must be serialised by the caller.  Like the other entry points it returns
 * FCC_ERR_TIMEOUT (and clears the plan's status word) when an earlier call
 * of the plan recorded a device-side timeout.
 */
#define FCC_STATIC_SCRATCH_BYTES (16u << 20)
fcc_status fcc_dct_inverse_static(fcc_plan* plan, const void* in, void* out, void* stream);

/*
 * Wait for the device (cudaDeviceSynchronize) and report a device-side
 * failure of the plan's earlier calls: FCC_ERR_TIMEOUT if a bounded wait of a
 * tensor-core kernel gave up (the kernel then skipped its remaining work and
 * released its tensor memory), FCC_ERR_CUDA if a launch or the device
 * failed.  Clears the plan's status word.  The word lives in pinned host
 * memory, so the plan's next forward / inverse / adjoint call also returns
 * FCC_ERR_TIMEOUT (without launching, and clearing it) once a kernel of an
 * earlier call has recorded a timeout.
 */
fcc_status fcc_dct_check(fcc_plan* plan);

/*
 * Test hook for the device-side failure detection (no counterpart in the
 * paper).  With enable != 0 the tensor-core kernels of a tensor-core plan
 * issue no MMA and no completion signal, so their bounded wait runs out after
 * a short limit (65536 non-blocking polls): the kernel records the
 * timeout, releases its tensor memory and returns without writing its
 * output, and the next fcc_dct_check reports FCC_ERR_TIMEOUT.  The GPU is
 * neither hung nor faulted; later calls with enable = 0 run normally.
 * FCC_ERR_UNSUPPORTED for plans without a tensor-core form.
 */
fcc_status fcc_dct_test_wait_timeout(fcc_plan* plan, int enable);

/*
 * Test hooks for host-side allocation failure (no counterpart in the paper;
 * nothing on the GPU is made to fail).  fcc_dct_test_fail_alloc(nth) arms a
 * one-shot failure: counting from the call, the nth allocation the library
 * makes in this process -- the plan object (host), the pinned status word, a
 * device table or workspace (plan creation, the first packed or host-buffer
 * call) -- reports failure instead, as an exhausted allocator would.  The
 * entry point that made it returns NULL (plans) or FCC_ERR_ALLOC after
 * releasing what it had allocated.  nth = 0 disarms; nth < 0 is
 * FCC_ERR_INVALID_ARG.  fcc_dct_test_allocations reports what the library
 * holds right now: the number of live plans and the device bytes they own
 * (through *plans and *device_bytes when not NULL); returns the number of
 * allocations made since the process started.
 */
fcc_status fcc_dct_test_fail_alloc(int nth);
int64_t fcc_dct_test_allocations(int64_t* plans, int64_t* device_bytes);

/*
 * Execution schedule.  The paper has no counterpart: these knobs change only
 * how the plan's work is laid out on the GPU (the results agree to FP32
 * rounding order).  Keys and values:
 *   FCC_SCHED_CHUNK_MB   1..1024   MB of complex intermediate per chunk of
 *                                  volumes (kept L2-resident between passes);
 *                                  inverse / adjoint chunks stay within the
 *                                  workspace sized at plan creation
 *   FCC_SCHED_STREAMS    1..4      internal streams the chunks alternate over
 *                                  (inverse / adjoint: at most the count at
 *                                  plan creation)
 *   FCC_SCHED_RAGGED     0, 1, 2   ragged FP32 forward: 0 = one mixing, slab and
 *                                  pencil launch per distinct order; 1 = the
 *                                  whole batch in one persistent cooperative
 *                                  launch (orders with a register-radix DFT,
 *                                  at most 16 distinct orders, else
 *                                  FCC_ERR_UNSUPPORTED); 2 = one launch set per
 *                                  run of equal orders
 *   FCC_SCHED_TC_BLOCKS  0..4      tensor-core mixing: blocks per SM in the
 *                                  grid (0 = as many as can be resident)
 *   FCC_SCHED_TC_FOLD    0, 1      tensor-core forward, orders with register
 *                                  DFT passes: 1 (default) = the mixing writes
 *                                  its sums without the row phase and 1/24
 *                                  (the slot's 8th-root wrap factor is in the
 *                                  core) and the slab / pencil passes multiply
 *                                  their inputs by the separable rest; 0 = the
 *                                  mixing applies the row phase
 * set_schedule returns FCC_ERR_INVALID_ARG for an unknown key or a value out
 * of range; get_schedule returns the current value, or -1 on a bad argument.
 */
typedef enum {
    FCC_SCHED_CHUNK_MB = 0,
    FCC_SCHED_STREAMS = 1,
    FCC_SCHED_RAGGED = 2,
    FCC_SCHED_TC_BLOCKS = 3,
    FCC_SCHED_TC_FOLD = 4
} fcc_sched_key;
fcc_status fcc_dct_set_schedule(fcc_plan* plan, int key, int value);
int fcc_dct_get_schedule(const fcc_plan* plan, int key);

/*
 * Autotuner (no counterpart in the paper): times the forward transform of
 * `in` into `out` (device buffers, the layouts of fcc_dct_forward) under the
 * candidate schedules -- chunk size (8, 16, 32, 64 MB) x internal streams
 * (1-4), then the tensor-core grid, for uniform plans; per-order launches x
 * streams, the persistent
 * launch and per-run launches for ragged plans -- with one untimed call and
 * `reps` (1..100) timed calls each, keeps the fastest and writes its time per
 * call to *best_ms (if not NULL).  Synchronises `stream`; overwrites `out`.
 * Candidates the device refuses are skipped.
 *
 * Cache: when the environment variable FCC_AUTOTUNE_CACHE names a file, the
 * result is appended to it as one JSON object per line, keyed by the order
 * (ragged plans: a hash of the order list), batch, dtype, shift and GPU name;
 * a later call for the same key applies the cached schedule, times it with
 * `reps` calls for *best_ms and skips the search (a cached schedule the
 * device refuses is searched again).  The file is advisory: if it is
 * missing, unreadable or malformed the search runs, and a failed write is
 * ignored.
 */
fcc_status fcc_dct_autotune(fcc_plan* plan, const void* in, void* out, void* stream, int reps, float* best_ms);

/* Status of the last failing call on this host thread (FCC_OK if none). */
fcc_status fcc_dct_last_error(void);
const char* fcc_status_string(fcc_status status);

/* Release the plan's device memory.  Accepts NULL. */
void fcc_dct_destroy(fcc_plan* plan);

/*
 * Host-only description of the orbit structure for order n (no CUDA calls;
 * usable without a GPU).  Fills, when the pointers are non-NULL:
 *   n_orbits, n_classes, free_class (-1 if none);
 *   reps[n_orbits]       packed representatives k1 | k2<<10 | k3<<20,
 *   cls[n_orbits]        class of each orbit,
 *   wrap[n_classes*72]   wrap vectors m_h (int8 as int32), slot-major,
 *   canon[n_classes*24]  canonical slot of each slot,
 *   fwd/inv/adj[n_classes*576*2]  24x24 complex cores (re, im) in double.
 * Call once with NULL arrays to learn the sizes.
 */
fcc_status fcc_dct_describe(int order, int64_t* n_orbits, int* n_classes, int* free_class,
                            uint32_t* reps, int32_t* cls, int32_t* wrap, int32_t* canon,
                            double* fwd, double* inv, double* adj);

/* The same for the skew transform of shift v / d (as fcc_dct_plan_skew);
 * *invertible (if non-NULL) is 1 when every class block is invertible, else
 * 0 (the inverse core of each singular class is then left zero). */
fcc_status fcc_dct_describe_skew(int order, const int* v, int d, int* invertible, int64_t* n_orbits,
                                 int* n_classes, int* free_class, uint32_t* reps, int32_t* cls, int32_t* wrap,
                                 int32_t* canon, double* fwd, double* inv, double* adj);

/*
 * Host-only description of the tiles the orbit-mixing kernels walk at order n
 * (no CUDA calls).  Fills, when the pointers are non-NULL: ntiles;
 * free_tiles (the free-class tiles come first); tile_off[ntiles + 1], the
 * offsets of the tiles in tile_reps; tile_reps[n_orbits], the packed
 * representatives (as in fcc_dct_describe) in tile order.  A tile holds at
 * most 32 orbits of one class.  Call once with NULL arrays to learn ntiles.
 */
fcc_status fcc_dct_describe_tiles(int order, int32_t* ntiles, int32_t* free_tiles, int32_t* tile_off,
                                  uint32_t* tile_reps);

/* The 24 group matrices (row-major 3x3 each) the library uses. */
fcc_status fcc_dct_weyl_group(int32_t* out /* 216 */);

#ifdef __cplusplus
}
#endif

#endif /* FCC_DCT_H */
