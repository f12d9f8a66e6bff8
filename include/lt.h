/*
 * lt.h -- C ABI of the GB300 lens-transport library (liblt.so).
 *
 * What it computes (Precomputed Lens Transport Maps, Sec. 3):
 *   the lens transport map T(p_in, w_in, I_in, lambda) -> {(p_out, w_out, I_out)}_k
 *   of Eq. 1, one path k at a time (Sec. 4.2 path decomposition), for a
 *   static, rotationally symmetric lens of spherical or planar surfaces under
 *   geometric optics.  A path's operator is the composition of per-surface
 *   operators S_{L,sigma} = (closest hit p_sigma, new direction d_{L,sigma},
 *   Fresnel factor f_{L,sigma}) (Eq. 5-7).  A ray is valid iff the last
 *   surface it reaches is the output (image) plane (Sec. 3).
 *
 * Conventions shared by every entry point:
 *   - Units: mm; wavelengths in nm (glass formulas use micrometres).
 *   - Frame: optical axis +z, light travels +z, entrance plane z = 0, surface
 *     1's vertex at prescription.entrance_gap.  Entrance rays are given by
 *     their point (x, y, 0) and direction (dx, dy, dz), dz > 0; the direction
 *     need not be exactly unit (it is normalised on load).
 *   - Ray arrays are structure-of-arrays FP32.  Unless an entry point says
 *     "host", pointers are DEVICE pointers on the current CUDA device, each
 *     array 16-byte aligned, and the call only enqueues work on `stream`:
 *     the caller keeps the buffers alive until the stream has passed the
 *     work.  The library never frees caller memory.
 *   - Errors: every lt_status call returns LT_OK (0) or a negative code and
 *     leaves a message for lt_last_error() in the calling thread.  Nothing
 *     throws across this boundary.  Per-ray problems never fail a call: they
 *     go into the ray's flags byte (LT_FLAG_*), and an invalid ray has all
 *     six outputs set to 0.
 *   - Paths: path_id 0 is the transmission path through surfaces 1..S;
 *     path_id 1 .. S(S-1)/2 are the two-bounce ghosts (i, j), 1 <= i < j <= S,
 *     numbered lexicographically ((1,2) = 1, (1,3) = 2, ...).  A ghost goes
 *     forward 1..j reflecting at j, back j-1..i reflecting at i, then
 *     forward i+1..S to the image plane (Sec. 4.2: paths with more than two
 *     reflections are dropped).
 */
#ifndef LT_H
#define LT_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef int lt_status;
#define LT_OK          0
#define LT_EINVAL     -1   /* bad argument (NULL, size, alignment, path id) */
#define LT_ENOMEM     -2   /* device or host allocation failed */
#define LT_ECUDA      -3   /* a CUDA runtime call failed */
#define LT_EBUSY      -4   /* resource in use */
#define LT_ETIMEOUT   -5   /* a bounded wait ran out */
#define LT_ENOTREADY  -6   /* work not finished yet */
#define LT_EBADLENS   -7   /* prescription rejected */
#define LT_EIO        -8   /* file read/write failed */

/* A cudaStream_t (same type, no CUDA header needed); NULL = legacy default stream. */
typedef struct CUstream_st* lt_stream;

/* ------------------------------------------------------------------ lenses */

#define LT_MAX_SURFACES 32
#define LT_MAX_GLASSES  32

enum { LT_GLASS_AIR = 0, LT_GLASS_CAUCHY = 1, LT_GLASS_SELLMEIER = 2 };
enum { LT_IMAGE_PARAXIAL = 0, LT_IMAGE_ABS = 1 };

/* Dispersion (the paper takes lambda as an input everywhere, Eq. 1-2):
 * Cauchy n = A + B / lam^2, Sellmeier n^2 = 1 + sum_i B3[i] lam^2 / (lam^2 - C3[i]),
 * lam in micrometres. */
typedef struct {
    int kind;
    double A, B;
    double B3[3], C3[3];
} lt_glass;

typedef struct {
    double curvature;    /* 1/R (1/mm); 0 = plane; > 0: centre of curvature on the +z side */
    double thickness;    /* vertex to next vertex (mm); ignored for the last surface */
    double aperture_r;   /* clear aperture radius (mm): a hit with x^2+y^2 > r^2 is absorbed */
    int glass_after;     /* index into glasses[] of the medium after this surface; -1 = air */
    /* Even asphere (the circularly symmetric surfaces Sec. 4.1 admits): sag
     * z(r) = c r^2 / (1 + sqrt(1 - (1 + conic) c^2 r^2)) + A4 r^4 + A6 r^6 + A8 r^8
     * + A10 r^10 in the vertex frame; all zero: the sphere (or plane).  A lens
     * with an asphere is traced by Newton's method on the sag (FP32) from the
     * base sphere's hit, on the tracer's general instantiation. */
    double conic;
    double asph[4];      /* A4, A6, A8, A10 (1/mm^3, 1/mm^5, ...) */
} lt_surface;

typedef struct {
    int n_surfaces;              /* 1 .. LT_MAX_SURFACES */
    const lt_surface* surfaces;  /* host array, copied by lt_create_lens */
    int n_glasses;               /* 0 .. LT_MAX_GLASSES */
    const lt_glass* glasses;     /* host array, copied */
    double entrance_gap;         /* entrance plane (z = 0) to the vertex of surface 1 */
    int stop_after;              /* aperture stop in the gap after this surface (0: in front of 1) */
    double stop_offset;          /* stop plane z relative to that gap's start (z = 0 or vertex) */
    double stop_r;               /* stop radius; <= 0: no stop */
    int image_mode;              /* LT_IMAGE_PARAXIAL: paraxial focus at lambda_ref_nm;
                                    LT_IMAGE_ABS: the plane z = image_z */
    double image_z;
    double lambda_ref_nm;        /* reference wavelength of the paraxial focus (e.g. 587.6) */
    double edge_eps_mm;          /* near-edge flag band; <= 0 selects 1e-6 mm */
    double grazing_k;            /* ill-conditioning band on k = 1 - eta^2 sin^2 i; <= 0 selects 1e-2 */
} lt_prescription;

typedef struct lt_lens lt_lens;

/* Validate and copy a prescription, compute the image plane (paraxial
 * ABCD product in FP64 when image_mode is LT_IMAGE_PARAXIAL) and stage the
 * lens for the kernels.  Medium after the last surface is forced to air.
 * Errors: LT_EINVAL (NULL / counts out of range), LT_EBADLENS (glass index
 * out of range, aperture larger than a sphere, back focal distance <= 0).
 * The caller owns *out and releases it with lt_destroy_lens. */
lt_status lt_create_lens(const lt_prescription* p, lt_lens** out);
void lt_destroy_lens(lt_lens* lens);

/* The lens seen from its image side, for backward path tracing (Sec. 3,
 * Eq. 9: rays leave the sensor, cross the lens in reverse along the full
 * transmission path and go on into the scene).  The backward transport of
 * the lens is the forward transport of its mirror image about the sensor
 * plane z = sensor_z (absolute z of the forward lens): surface j of the new
 * lens is forward surface S + 1 - j with negated curvature, the same clear
 * aperture and the media shifted; the stop keeps its plane; the new lens's
 * entrance plane is the sensor and its image plane (LT_IMAGE_ABS) the
 * forward plane z = out_z in front of surface 1.  In its frame z' =
 * sensor_z - z, a ray leaving the sensor at (x, y) along the forward
 * direction (dx, dy, -dz), dz > 0, is the entrance ray (x, y, dx, dy, dz),
 * and an exit ray (x', y', dx', dy', dz') is the forward ray at z = out_z
 * along (dx', dy', -dz').  Every other call (lt_trace, lt_build_map,
 * lt_mlp_train, ...) applies to the result unchanged, so the backward map of
 * the paper's depth-of-field rendering is a map of the reversed lens.  Moving
 * sensor_z refocuses (the paper's manual focusing).
 * Errors: LT_EINVAL (NULL, a sensor plane not behind the last surface's cap,
 * an output plane behind the first surface's cap, or a stop outside the two
 * planes), or those of lt_create_lens.  The caller owns *out. */
lt_status lt_reverse_lens(const lt_lens* lens, double sensor_z, double out_z, lt_lens** out);

/* Paraxial data of a lens at lambda_nm (host, FP64): effective focal length,
 * back focal distance, and the image-plane z in use.  Any output may be NULL. */
lt_status lt_lens_paraxial(const lt_lens* lens, double lambda_nm, double* efl, double* bfd,
                           double* z_image);

/* Number of paths of the lens (1 + S(S-1)/2) and the (i, j) of a path id. */
int32_t lt_lens_n_paths(const lt_lens* lens);
lt_status lt_path_ij(int32_t n_surfaces, int32_t path_id, int32_t* i, int32_t* j);
/* Path id of ghost (i, j) (0 for i = j = 0), or -1 if out of range. */
int32_t lt_path_id(int32_t n_surfaces, int32_t i, int32_t j);
/* Paper-style binary path code (Fig. 2 caption; values in Fig. 7): bit k-1 is
 * set when interaction k reflects (first interaction = least significant
 * bit), plus a leading 1 at bit K, K = number of interactions.  0 on error. */
uint64_t lt_path_code(int32_t n_surfaces, int32_t i, int32_t j);

/* ------------------------------------------------------------------ rays */

/* Ray flags (one byte per ray). */
#define LT_FLAG_VALID      0x01  /* reached the image plane */
#define LT_FLAG_NEAR_EDGE  0x02  /* some aperture/stop test was within edge_eps_mm of its edge */
#define LT_FLAG_NEAR_TIR   0x04  /* some interaction had |1 - eta^2 sin^2 i| < 1e-6 */
#define LT_FLAG_BAD_INPUT  0x08  /* NaN/Inf input, dz <= 0 or lambda <= 0 */
#define LT_FLAG_TRACED     0x10  /* a map query answered this ray with the exact tracer */
#define LT_FLAG_OUTSIDE    0x20  /* a map query found the ray outside the map's lattice box */
#define LT_FLAG_GRAZING    0x40  /* some interaction had 0 <= k < grazing_k: the ray left within
                                    ~6 deg of grazing and its FP32 output error is amplified by
                                    ~1/(2 sqrt k) (ill-conditioned, reported separately) */

typedef struct {
    const float *x, *y;          /* entrance point on z = 0 */
    const float *dx, *dy, *dz;   /* entrance direction */
} lt_rays_in;

typedef struct {
    float *x, *y;                /* exit point on the image plane */
    float *dx, *dy, *dz;         /* exit direction (unit) */
    float *I;                    /* Fresnel throughput I_out for I_in = 1 */
    uint8_t* flags;              /* LT_FLAG_* */
} lt_rays_out;

/* Brute-force FP32 trace of n rays along one path (Sec. 3, Eq. 6-7).
 * in/out/lambda_nm: device arrays of n entries.  Paths of more than 4
 * interactions run as two kernels per wave of at most 2^24 rays: one thread
 * per ray through the first three interactions (where most rays of a lens
 * die), then the survivors, queued, in dense warps to the end; the queue
 * (54 B per ray of the wave) is taken stream-ordered from the library's
 * memory pool.  Shorter paths run as one kernel whose blocks compact their
 * surviving rays in shared memory.
 * Errors: LT_EINVAL (NULL pointer with n > 0, misaligned array, bad path id),
 * LT_ENOMEM (queue allocation), LT_ECUDA (launch failed).  n = 0 is a no-op. */
lt_status lt_trace(const lt_lens* lens, const lt_rays_in* in, const float* lambda_nm,
                   int32_t path_id, const lt_rays_out* out, size_t n, lt_stream stream);

/* Same, with HOST arrays (pageable or pinned; pinned is faster): traces in
 * pipelined chunks of about n / 8 rays (2^16 to 2^20) and returns when the
 * outputs are in host memory.  Each chunk passes through three library
 * streams (copy in, kernels, copy out), so one chunk's inputs copy in while
 * an older chunk's outputs copy back.  When the six input arrays lie at equal
 * distances in memory (rows of one block), each chunk's inputs move in one
 * strided copy, and likewise the six float outputs; otherwise one copy per
 * array.  Errors as lt_trace, plus LT_ENOMEM for staging buffers. */
lt_status lt_trace_host(const lt_lens* lens, const lt_rays_in* in, const float* lambda_nm,
                        int32_t path_id, const lt_rays_out* out, size_t n);

/* The tracer's own FP32 reciprocal and square root, element by element, so
 * that their accuracy can be checked against correctly rounded results.
 * Every interaction of lt_trace (Sec. 3, Eq. 2-7) divides by the hit root's
 * denominator, by the index n2 of the medium entered and by the product of
 * the two Fresnel denominators, and takes two square roots; the tracer forms
 * each reciprocal as the hardware approximation plus one Newton-Raphson step
 * r' = r + r (1 - x r), and each square root from the hardware reciprocal
 * square root plus one Newton step.  Outputs: rcp[i] = 1 / x[i] (within about
 * 1 ulp for finite nonzero x[i] whose reciprocal is a normal number) and
 * sqrt_out[i] = sqrt(x[i]) (about 1 ulp for x[i] > 0; 0 for x[i] <= 0).
 * x, rcp, sqrt_out: DEVICE arrays of n floats owned by the caller; the
 * outputs must not overlap x.  Asynchronous on `stream`.  Errors: LT_EINVAL
 * for a NULL array with n > 0 or n above 2^38; LT_ECUDA if the launch fails.
 * n = 0 is a no-op. */
lt_status lt_tracer_math(const float* x, float* rcp, float* sqrt_out, size_t n, lt_stream stream);

/* Compacted output of lt_trace_paths: path p owns the segment
 * [p * capacity, (p + 1) * capacity) of every array.  Only rays that reach
 * the image plane are written, in no particular order within a segment. */
typedef struct {
    float *x, *y, *dx, *dy, *dz, *I;  /* as lt_rays_out, valid rays only */
    uint8_t* flags;                   /* LT_FLAG_* of each written ray (VALID always set) */
    uint32_t* ray_index;              /* which entrance ray (0..n-1) the entry belongs to */
    uint32_t* valid_count;            /* n_paths counters: rays of path p that reached the image */
    size_t capacity;                  /* entries per path segment (>= 1) */
} lt_paths_out;

/* Trace the same n entrance rays along n_paths paths in one launch (the flare
 * workload of Sec. 4.2: the main path plus every two-bounce ghost (i, j),
 * each ray's wavelength drawn per path).  path_ids: HOST array of n_paths ids
 * (duplicates allowed).  lambda_nm: device array; path p reads
 * lambda_nm[p * lambda_stride + r] (lambda_stride = 0: one wavelength array
 * for all paths).  Rays are compacted per path; valid_count[p] is set to the
 * true count even when it exceeds capacity, in which case only `capacity`
 * of them (which ones is unspecified) are written -- compare the count with
 * capacity after the stream synchronises.  Per-ray results are identical to
 * lt_trace of the same ray, path and wavelength.  The paths run in waves of
 * at most 2^24 (path, ray) pairs, each as two kernels: every ray through its
 * first three interactions, then the queued survivors to the end; the queue
 * (54 B per pair of a wave) comes stream-ordered from the library's pool.
 * Errors: LT_EINVAL (NULL pointer, misaligned array, n_paths < 1 or > 1024,
 * bad path id, capacity 0, n >= 2^32), LT_ENOMEM (queue allocation),
 * LT_ECUDA.  n = 0 zeroes the counters. */
lt_status lt_trace_paths(const lt_lens* lens, const lt_rays_in* in, const float* lambda_nm,
                         size_t lambda_stride, const int32_t* path_ids, int32_t n_paths,
                         const lt_paths_out* out, size_t n, lt_stream stream);

/* The sensor of forward light tracing: a width x height grid of square
 * pixels of side pixel_mm on the image plane, centred on the axis (pixel
 * (i, j) has its centre at ((i + 0.5 - width / 2) pixel_mm,
 * (j + 0.5 - height / 2) pixel_mm)), row-major images of floats. */
typedef struct {
    int32_t width, height;       /* pixels, 1..65536 */
    double pixel_mm;             /* pixel side, > 0 */
    float weight;                /* factor on every deposit (1 / n: the per-sample average) */
    int32_t per_path;            /* 0: one image, all paths summed; 1: one image per path */
} lt_sensor;

/* Forward light tracing onto the sensor (Sec. 3, Eq. 8): trace the n
 * entrance rays along n_paths paths exactly as lt_trace_paths does (same
 * waves, kernels and per-ray arithmetic) and add, for every ray that reaches
 * the image plane, I_out * G * h(x_out - c) * weight to each pixel c, with
 * G = d_z of the exit direction (its cosine to the sensor normal) and h the
 * tent (bilinear) pixel filter of one pixel radius -- the paper names no
 * filter.  Deposits are FP32 atomic adds (their order, and so the last bits
 * of a pixel, varies between runs).  image: DEVICE float[per_path ? n_paths
 * : 1][height][width], 16-byte aligned, accumulated into (the caller clears
 * it).  path_ids, lambda_nm and lambda_stride as lt_trace_paths.  Rays that
 * land outside the sensor deposit nothing there.  Errors: LT_EINVAL (NULL or
 * misaligned pointer, bad sensor, n_paths < 1 or > 1024, bad path id,
 * n >= 2^32), LT_ENOMEM (queue allocation), LT_ECUDA. */
lt_status lt_splat_paths(const lt_lens* lens, const lt_rays_in* in, const float* lambda_nm,
                         size_t lambda_stride, const int32_t* path_ids, int32_t n_paths, size_t n,
                         const lt_sensor* sensor, float* image, lt_stream stream);

/* ------------------------------------------------------------------ valid-region sampling */

/*
 * The sampler the paper uses to gather training rays (Sec. 5.1, data
 * collection): for most paths only a small fraction of the input space gives
 * valid rays, so Markov chains with the path's binary visibility as target
 * draw rays uniformly over the valid region.  A chain lives in the box
 * [lo, hi] over (x, y, s_x, s_y, lambda); its ray is (x, y) with direction
 * normalize(s_x, s_y, 1).  It starts at the first valid independent uniform
 * draw (at most init_tries; a chain that finds none never starts), then
 * each step proposes, with probability p_large, an independent uniform
 * point, else a uniform point of the box of half-width small * (hi - lo)
 * around its state, and moves iff the proposal is in the box and its ray is
 * valid (the exact FP32 tracer decides).  Random numbers are counter-based:
 * u(chain, i, k) = top 24 bits of SplitMix64(seed + (chain << 32 | i << 3 |
 * k)) * 2^-24, i the init try t or init_tries + step, k 0 for the step kind
 * and 1..5 for the dimensions; every proposal is computed in FP32 with one
 * rounding per operation, so the samples are a pure function of the options.
 */
typedef struct {
    int32_t path_id;
    double lo[5], hi[5];          /* the box over (x, y, s_x, s_y, lambda) */
    uint64_t seed;
    int32_t chains, steps;        /* chains x steps samples, < 2^32 */
    double small;                 /* small-step half-width, as a fraction of the box */
    double p_large;               /* probability of an independent step, in [0, 1] */
    int32_t init_tries;           /* >= 1; init_tries + steps < 2^29 */
} lt_mcmc_opts;

typedef struct {
    float *x, *y, *dx, *dy, *dz;  /* device, chains x steps: the entrance ray of sample */
    float* lambda_nm;             /* (step s, chain c) at index s * chains + c */
    uint8_t* flags;               /* LT_FLAG_VALID for a started chain's samples; 0 (and zero rays) otherwise */
    uint32_t* accepted;           /* device, per chain: proposals accepted (may be NULL) */
} lt_samples_out;

/* Run the chains (one GPU thread per chain) and write every chain's state
 * after every step.  The samples feed lt_build_map (fit rays) or
 * lt_mlp_train like any rays.  Errors: LT_EINVAL (NULL or misaligned array,
 * bad path id, empty box, counts out of range), LT_ECUDA. */
lt_status lt_mcmc_sample(const lt_lens* lens, const lt_mcmc_opts* opts, const lt_samples_out* out,
                         lt_stream stream);

/* ------------------------------------------------------------------ maps */

/*
 * Precomputed lens transport map of one path (Sec. 4, "Precomputed Lens
 * Transport Maps"): the factorised form of Sec. 4.2 -- a binary valid/occluded
 * mask (Eq. 11: output f(x) if g(x) = 1, nothing otherwise) and a regressor
 * used only on unblocked rays.  Here the regressor is a table:
 *   - a regular lattice over the 5-D input box (x, y, s_x, s_y, lambda) with
 *     s = (d_x/d_z, d_y/d_z) the entrance direction slopes; every node is
 *     traced exactly (FP32, the lt_trace tracer); node layout row-major over
 *     (x, y, s_x, s_y, lambda), lambda fastest, 6 floats per node
 *     (x, y, dx, dy, dz, I at the image plane; zeros if the node is invalid);
 *   - every cell is INVALID (its 32 corners and every fit ray inside it are
 *     invalid), VALID (all corners and fit rays valid, and no fit ray's exit
 *     position differs from interpolation by more than max_residual_mm) or
 *     BOUNDARY (anything else), 2 bits per cell;
 *   - a query answers a VALID cell by multilinear interpolation of its 32
 *     corners (direction renormalised), an INVALID cell with "no output", and
 *     a BOUNDARY cell -- or a ray outside the box -- with the exact tracer
 *     (the tracer is the map's fallback near mask boundaries).
 * The cell of a ray is decided in FP32 with correctly rounded operations, in
 * this order: s = d_x / d_z; u = (v - lo) * inv_step; cell = min(floor(u),
 * res - 2); inside iff 0 <= u <= res - 1 on every axis; lo, step and
 * inv_step are the FP32 roundings of lo, (hi - lo)/(res - 1) and its inverse.
 * Node entrance rays are built the same way: q = lo + i * step (each step
 * rounded), d = (s_x, s_y, 1) / sqrt(s_x^2 + s_y^2 + 1).
 */
typedef struct lt_map lt_map;

typedef struct {
    int32_t path_id;             /* path the map represents */
    int32_t res[5];              /* nodes along x, y, s_x, s_y, lambda; each >= 2 */
    double lo[5], hi[5];         /* lattice box (mm, mm, slope, slope, nm) */
    double max_residual_mm;      /* <= 0: no limit; else VALID cells also need every fit
                                    ray's |interpolated - traced| exit position <= this */
    const float *fit_x, *fit_y, *fit_dx, *fit_dy, *fit_dz, *fit_lambda;  /* device arrays */
    size_t n_fit;                /* fit rays (may be 0: classes from corners alone) */
    int32_t node_format;         /* LT_NODE_F32 (0) or LT_NODE_S16 */
} lt_map_opts;

/* Node table formats (Sec. 4.2's regressor as a table).  LT_NODE_F32: six
 * FP32 outputs per node in a 32-byte record.  LT_NODE_S16: the half-size
 * table -- output k of a node is a 16-bit integer q times step_k =
 * 2^(e_k - 15), 2^e_k the smallest power of two above the largest |value| of
 * output k over the valid nodes, q the FP32 node value times 2^(15 - e_k)
 * rounded to nearest (ties to even), invalid nodes 0; 16-byte records
 * (6 x int16 + 4 bytes of padding), so a cell's lambda-adjacent pair of
 * corners is one 32-byte sector.  A query interpolates the integers in FP32
 * and multiplies by step_k, so it differs from interpolating the FP32 nodes
 * by at most step_k / 2 before the direction is renormalised.  The class
 * certification (max_residual_mm) is made on the FP32 nodes. */
enum { LT_NODE_F32 = 0, LT_NODE_S16 = 1 };

typedef struct {
    uint64_t n_nodes, n_cells, valid_nodes;
    uint64_t cells_invalid, cells_valid, cells_boundary;
    uint64_t fit_inside, fit_valid;          /* fit rays inside the box / valid */
    double fit_residual_rms_mm;              /* over valid fit rays in cells whose corners are all valid */
    double fit_residual_max_mm;
    uint64_t table_bytes;                    /* device bytes held by the map */
    double build_ms;                         /* wall time of lt_build_map */
    int32_t node_format;                     /* LT_NODE_* */
    float node_step[6];                      /* LT_NODE_S16: step_k of each output; else 0 */
} lt_map_stats;

/* Build a map on the current device: trace the lattice nodes, trace and
 * reduce the fit rays per cell (FP64 residual sums), classify the cells.
 * Work runs on `stream`; the call returns when the map is complete.  The map
 * keeps a copy of the lens (no reference to `lens`).  Errors: LT_EINVAL
 * (resolution < 2, empty box, bad path, misaligned fit arrays), LT_ENOMEM,
 * LT_ECUDA.  The caller releases *out with lt_destroy_map. */
lt_status lt_build_map(const lt_lens* lens, const lt_map_opts* opts, lt_map** out,
                       lt_stream stream);
void lt_destroy_map(lt_map* map);
lt_status lt_map_stats_get(const lt_map* map, lt_map_stats* out);

enum {
    LT_QUERY_TABLE = 0,        /* mask + table, exact tracer for BOUNDARY cells (default) */
    LT_QUERY_NO_MASK = 1       /* ablation of Fig. 6: ignore the mask, interpolate every ray
                                  inside the box over all 32 corners (invalid nodes count as
                                  zeros) and report it valid; outside the box: tracer */
};

/* Query the map for n rays (device arrays, as lt_trace): the factorised
 * lookup of Sec. 4.2 (Eq. 11).  A table map: a first kernel classifies every
 * ray, answers INVALID cells, interpolates VALID cells and queues BOUNDARY
 * cells and rays outside the box; a second traces the queue exactly (those
 * rays carry LT_FLAG_TRACED) and writes their results.  A polynomial-patch
 * map: the first kernel classifies, queues and sorts the answered rays by
 * patch; the second evaluates their polynomials and then traces the queue.
 * The queue (28 bytes per ray; with a polynomial-patch map also a 32-byte
 * record per answered ray) comes from the library's stream-ordered memory
 * pool, which keeps freed blocks for reuse, so steady-state calls do not
 * reach cudaMalloc.
 * Batches of at most 2^18 rays run as one kernel whose blocks trace their
 * own queued rays (no queue, no pool); the results are the same either way.
 * Errors as lt_trace; LT_ENOMEM if the queue cannot be had; LT_EINVAL if the
 * current device is not the one the map was built or loaded on (this holds
 * for every call that takes a map). */
lt_status lt_query(const lt_map* map, const lt_rays_in* in, const float* lambda_nm,
                   const lt_rays_out* out, size_t n, int32_t mode, lt_stream stream);
/* Same with HOST arrays, in the pipelined chunks of lt_trace_host; returns
 * when the results are in host memory. */
lt_status lt_query_host(const lt_map* map, const lt_rays_in* in, const float* lambda_nm,
                        const lt_rays_out* out, size_t n, int32_t mode);

/* Map query that allocates nothing, for callers that cannot allocate GPU
 * memory while they run: a renderer or serving process whose own allocator
 * reserves the whole device at start-up (so a later cudaMalloc or pool
 * growth fails), or a loop where cudaMalloc and the device-wide
 * synchronisation it can imply are not allowed.  The paper has no
 * counterpart: this is a deployment aid.
 * Same arguments, results and errors as lt_query, but its trace queue lives
 * in a fixed array inside the library (28 bytes per ray of
 * LT_NOALLOC_MAX_RAYS rays after 8,448 bytes of counters: 14 MiB, held on
 * every device that loads the library until the process exits), so
 * n > LT_NOALLOC_MAX_RAYS is rejected with LT_EINVAL: split larger batches.
 *  - Every call looks up the array's device address on the current device
 *    (a driver query, no allocation; the first one on a device may load the
 *    library's device code there), so make the first call before any stream
 *    capture.  The library's device arrays do not survive a device reset:
 *    maps built before one must be rebuilt.
 *  - Every call shares the one array, and its counters are cleared on the
 *    call's stream: calls whose work overlaps on the GPU (different streams
 *    without an event between them) race and give wrong results.  Order
 *    them on one stream.
 *  - While the library's profiler is on (lt_profile_enable), each launch
 *    also records two CUDA events that the profiler creates; leave it off
 *    where nothing may be created during the call. */
#define LT_NOALLOC_MAX_RAYS (1 << 19)
lt_status lt_query_noalloc(const lt_map* map, const lt_rays_in* in, const float* lambda_nm,
                           const lt_rays_out* out, size_t n, int32_t mode, lt_stream stream);

/*
 * Polynomial-patch map of one path: the same factorised form (Sec. 4.2,
 * Eq. 11), over the symmetry-reduced input of Sec. 4.1 (Eq. 10), with the
 * regressor a least-squares polynomial per patch.
 *   - Reduced input of an entrance ray (x, y, d) at lambda (nm): slopes
 *     s = d_xy / d_z; r = |(x, y)|; (c, s') = (x, y) / r, or (1, 0) at r = 0;
 *     p = c s_x + s' s_y, q' = c s_y - s' s_x, mirror m = -1 if q' < 0 else 1,
 *     q = |q'|; w = (1000 / lambda)^2 (1/um^2, in which a Cauchy index is
 *     affine).  u = (r, p, q, w) lies in the box [0, rho] x [-smax, smax] x
 *     [0, smax] x [(1000/lam_hi)^2, (1000/lam_lo)^2]; the reduced ray is
 *     (r, 0) with direction normalize(p, q, 1).
 *   - Regressor: the box is split into patches[k] equal patches per axis; on
 *     a patch the exit (x', y', d_x', d_y', I) of the reduced ray is a
 *     polynomial of total degree `degree` in the patch-local xi = 2 (u - lo)
 *     / h - 1, whose coefficients minimise the squared error over a tensor
 *     grid of `samples` Chebyshev nodes cos(pi (k + 1/2) / samples) per axis,
 *     traced (FP32) through the UNCLIPPED lens -- the same surfaces and path
 *     with every clear aperture and the stop removed -- and solved by FP64
 *     normal equations (FP64 reductions, Cholesky) on the GPU.  Apertures
 *     decide only whether a ray passes, not where it goes, so this function
 *     is smooth across the vignetting edge and the mask carries the occlusion.
 *     A patch with fewer valid samples than terms, or a singular system, has
 *     no fit (its cells are BOUNDARY).
 *   - Mask: a class grid of patches[k] * cells[k] cells per axis whose nodes
 *     are traced through the real lens: INVALID (16 corners invalid and no
 *     valid fit ray inside), VALID (16 corners valid, the patch fitted, every
 *     corner's and fit ray's exit position within max_residual_mm of the
 *     polynomial's) or BOUNDARY, 2 bits per cell.
 *   - Query (lt_query and every call that takes a map): VALID -> the
 *     polynomial (FP32 Horner) at the ray's xi, d_z' = sqrt(1 - d_x'^2 -
 *     d_y'^2), mirrored and rotated back; INVALID -> no output; BOUNDARY or
 *     outside the box -> the exact tracer.  LT_QUERY_NO_MASK answers every ray
 *     inside the box whose patch has a fit with the polynomial.
 * The cell of a ray is decided in FP32 with correctly rounded operations in
 * this order: i_z = 1 / d_z; s_x = d_x * i_z, s_y = d_y * i_z; r = sqrt(x*x +
 * y*y); i_r = 1 / r; c = x * i_r, s' = y * i_r; p = c*s_x + s'*s_y; q' =
 * c*s_y - s'*s_x; t = 1000 / lambda;
 * w = t*t; g_k = (u_k - lo_k) * inv_k with lo_k, inv_k = C_k / (hi_k - lo_k)
 * the FP32 roundings; cell_k = min(floor(g_k), C_k - 1); inside iff 0 <= g_k
 * <= C_k.  Class-grid node i is the ray of v = lo + i * step (step_k the FP32
 * rounding of (hi_k - lo_k) / C_k): x = v_r, y = 0, n2 = (p*p + q*q) + 1,
 * len = sqrt(n2), d = (p / len, q / len, 1 / len), lambda = 1000 / sqrt(w).
 */
typedef struct {
    int32_t path_id;
    double rho;                  /* entrance radius bound (mm) */
    double smax;                 /* slope bound: p in [-smax, smax], q in [0, smax] */
    double lam_lo, lam_hi;       /* wavelength range (nm) */
    int32_t degree;              /* total degree of every patch polynomial, 1..LT_POLY_MAX_DEGREE */
    int32_t patches[4];          /* patches along (r, p, q, w), each >= 1 */
    int32_t cells[4];            /* mask cells per patch along each axis, each >= 1 */
    int32_t samples;             /* Chebyshev samples per axis and patch, degree + 1 .. 8 */
    double max_residual_mm;      /* <= 0: no limit */
    const float *fit_x, *fit_y, *fit_dx, *fit_dy, *fit_dz, *fit_lambda;  /* device; may be absent */
    size_t n_fit;                /* extra traced rays that can only demote cells to BOUNDARY */
} lt_poly_opts;

#define LT_POLY_MAX_DEGREE 5

typedef struct {
    uint32_t patches, patches_fit, terms;
    uint64_t samples_traced, samples_valid;
    double sample_residual_max_mm;   /* largest |fit - traced| exit position over valid samples */
    double corner_residual_max_mm;   /* over the corners of cells whose 16 corners are valid */
} lt_poly_stats;

/* Build a polynomial-patch map on the current device (see above).  Work runs
 * on `stream`; the call returns when the map is complete.  lt_map_stats_get
 * reports its mask (n_nodes: class-grid nodes; cells; fit rays, whose
 * residuals are taken against the FP32 polynomial as queried), and
 * lt_poly_stats_get the fit.  Errors: LT_EINVAL (bad option, empty box, bad
 * path, misaligned fit arrays, more than 2^31 nodes), LT_ENOMEM, LT_ECUDA.
 * The caller releases *out with lt_destroy_map. */
lt_status lt_build_poly_map(const lt_lens* lens, const lt_poly_opts* opts, lt_map** out,
                            lt_stream stream);
/* LT_EINVAL for a table map. */
lt_status lt_poly_stats_get(const lt_map* map, lt_poly_stats* out);
/* Copy a polynomial-patch map's fit to host memory: coef (patches x terms x 5
 * doubles, outputs x', y', d_x', d_y', I, patches row-major over (r, p, q, w)),
 * exps (terms x 4 exponents of (xi_r, xi_p, xi_q, xi_w), in the order of
 * coef's terms), patch_ok (patches bytes).  Any pointer may be NULL.
 * LT_EINVAL for a table map. */
lt_status lt_poly_export(const lt_map* map, double* coef, int32_t* exps, uint8_t* patch_ok);

/* Copy the map to host memory for inspection: node6 (n_nodes x 6 floats; a
 * table map only, NULL for a polynomial-patch map; an LT_NODE_S16 table gives
 * its decoded values q * step), node_valid (n_nodes
 * bytes, 1/0), cell_class (n_cells bytes: 0 INVALID, 1 VALID, 2 BOUNDARY;
 * cells and nodes row-major over the map's axes, the last fastest).  Any
 * pointer may be NULL. */
lt_status lt_map_export(const lt_map* map, float* node6, uint8_t* node_valid,
                        uint8_t* cell_class);

/* Persist a map (lattice, tables, classes, the lens it was built on) to a
 * file, and load it back onto the current device.  Table maps with an
 * LT_NODE_F32 table only (LT_EINVAL otherwise).  Errors: LT_EIO. */
lt_status lt_map_save(const lt_map* map, const char* path);
lt_status lt_map_load(const char* path, lt_map** out);

/* ------------------------------------------------------------------ learned maps */

/*
 * The paper's learned form of a path's map (Sec. 4.2, Sec. 5.1): a binary
 * classifier g (4 -> 32 -> 32 -> 1, tanh hidden, logit out) and a regressor f
 * (4 -> 32 x 5 -> 6, tanh hidden, linear out); a ray gets f(x) iff g(x) > 0
 * (Eq. 11).  Inputs are the symmetry-reduced entrance ray of Sec. 4.1 (Eq. 10):
 * rotate about the axis so the point is (r, 0), mirror y if the rotated d_y < 0;
 * x = (2 r / rho - 1, d_x' / wmax, 2 d_y' / wmax - 1, 2 (lam - lam_lo) /
 * (lam_hi - lam_lo) - 1).  Regressor outputs are the exit (x', y'), direction
 * and throughput in the same reduced frame, standardised by the training set's
 * mean and standard deviation; a query mirrors and rotates them back.
 *
 * Parameter layout (FP32, flat, per network): for each layer in order the
 * weight matrix W (out x in, row-major) then the bias (out).
 * LT_MLP_REG_PARAMS = 4582, LT_MLP_CLS_PARAMS = 1249.
 */
#define LT_MLP_REG_PARAMS 4582
#define LT_MLP_CLS_PARAMS 1249

typedef struct lt_mlp lt_mlp;

typedef struct {
    int32_t path_id;
    double rho, wmax;               /* input box: r in [0, rho], |d_xy| <= wmax */
    double lam_lo, lam_hi;          /* wavelength range (nm) */
} lt_mlp_frame;

typedef struct {
    lt_mlp_frame frame;
    const float *fit_x, *fit_y, *fit_dx, *fit_dy, *fit_dz, *fit_lambda;  /* device training rays */
    size_t n_fit;
    const float* init_reg;          /* host: initial regressor parameters (the random draw is an input) */
    const float* init_cls;          /* host: initial classifier parameters */
    int32_t reg_steps, reg_batch;   /* regressor: Adam steps and rays per batch (valid rays only) */
    int32_t cls_steps, cls_batch;   /* classifier: steps and batch (all rays) */
    double lr, lr_decay;            /* schedule lr * lr_decay^(step / decay_every) (Sec. 5.1) */
    int32_t decay_every;
    int32_t ft_steps, ft_batch;     /* optional regressor fine-tune phase (0 steps: none) */
    double ft_lr;
    uint64_t seed;                  /* batch draws: SplitMix64(seed + step * batch + i) mod n */
    /* 0: every fit ray is a uniform draw of the input box.  Otherwise the
     * first n_fit_uniform rays are uniform draws and the rest are samples of
     * the path's valid region (lt_mcmc_sample), whose extra valid rays raise
     * the odds of "valid" in the classifier's training set by
     * k = 1 + (valid rays after the prefix) / (valid rays in the prefix); the
     * trained classifier's output bias is lowered by ln k so that its logit
     * answers for uniformly drawn rays (the prior-shift correction of a
     * calibrated classifier).  The regressor learns from every valid ray. */
    uint64_t n_fit_uniform;
} lt_mlp_opts;

typedef struct {
    uint64_t n_train, n_valid;      /* training rays traced, of which valid */
    double reg_loss, cls_loss;      /* mean training loss of the last 100 steps */
    double t_mean[6], t_std[6];     /* target standardisation */
    double train_ms;
    uint64_t tc_wait_timeouts;      /* tensor-core query waits that ran out (0 when healthy) */
    uint64_t n_valid_uniform;       /* valid rays among the first n_fit_uniform (all fit rays when 0) */
    double cls_prior_shift;         /* ln k subtracted from the classifier's output bias (0: none) */
} lt_mlp_stats;

enum {
    LT_MLP_F32 = 0,      /* FP32 SIMT, rational tanh (Lambert continued fraction, 9/10) */
    LT_MLP_BF16 = 1,     /* BF16 tensor-core MMA, FP32 accumulation, tanh.approx.bf16x2 */
    LT_MLP_F16 = 2,      /* FP16 tensor-core MMA, FP32 accumulation, tanh.approx.f16x2 */
    LT_MLP_F32_NOCLS = 3 /* ablation of Fig. 6: FP32 regressor for every ray, classifier off */
};

/* Trace the training rays (path frame.path_id), standardise the targets and
 * train both networks with Adam on the GPU (forward, backward and update are
 * this library's kernels; gradients are summed per block in FP32 and across
 * blocks in FP64).  Returns when training is done. */
lt_status lt_mlp_train(const lt_lens* lens, const lt_mlp_opts* opts, lt_mlp** out, lt_stream stream);

/* A learned map from given parameters (host FP32 arrays) and target
 * standardisation (6 means, 6 standard deviations). */
lt_status lt_mlp_create(const lt_lens* lens, const lt_mlp_frame* frame, const float* reg,
                        const float* cls, const double* t_mean, const double* t_std, lt_mlp** out);
void lt_destroy_mlp(lt_mlp* mlp);
lt_status lt_mlp_stats_get(const lt_mlp* mlp, lt_mlp_stats* out);
/* Copy the current parameters to host arrays (either may be NULL). */
lt_status lt_mlp_get_params(const lt_mlp* mlp, float* reg, float* cls);

/* Query n rays (device arrays as lt_trace) with LT_MLP_* arithmetic. */
lt_status lt_mlp_query(const lt_mlp* mlp, const lt_rays_in* in, const float* lambda_nm,
                       const lt_rays_out* out, size_t n, int32_t precision, lt_stream stream);

/* One forward and backward pass on an explicit batch with the current
 * parameters: net 0 = regressor (targets: B x 6 standardised, device), 1 =
 * classifier (targets: B labels 0/1 as floats, device); X: B x 4 network
 * inputs (device).  grad (host, FP64, the net's parameter count) receives the
 * gradient of the batch-mean loss, *loss the loss.  Synchronous. */
lt_status lt_mlp_grad(const lt_mlp* mlp, int32_t net, const float* X, const float* targets,
                      int32_t B, double* grad, double* loss);

/* Network inputs of n entrance rays (n x 4 device array out), as the query
 * and training kernels compute them (FP32). */
lt_status lt_mlp_features(const lt_mlp* mlp, const lt_rays_in* in, const float* lambda_nm,
                          float* X, size_t n, lt_stream stream);

/* ------------------------------------------------------------------ serving */

/*
 * A request server over one GPU: callers submit trace / map-query / learned-
 * map requests from any thread and poll tickets.  A native worker thread
 * launches them in arrival order on a few streams:
 *   - continuous batching: the small requests on device buffers waiting at
 *     the same time (n <= fuse_max_rays) run as one fused launch per kind
 *     whose request table is a kernel parameter, each block serving one
 *     request: TRACE requests of any lens and path together; QUERY requests
 *     of table maps (by query mode and dispersion form) and of
 *     polynomial-patch maps (LT_QUERY_TABLE, by degree and dispersion form);
 *     MLP requests by precision.  Per-ray results are identical to the same
 *     request made alone (lt_trace, lt_query, lt_mlp_query);
 *   - memory admission: a request holds device bytes while in flight (host
 *     staging 49 B/ray; a trace launched on its own also holds the tracer's
 *     queue of surviving rays, 54 B/ray of a wave of at most 2^24 rays); a
 *     request waits while
 *     the in-flight total would exceed mem_budget_bytes (one request alone is
 *     always admitted if it fits the budget, else lt_submit fails LT_ENOMEM);
 *   - deadlines: a request not launched within deadline_us of submission
 *     completes with LT_ETIMEOUT without running;
 *   - completion is signalled by a host function on the request's stream, so
 *     latency (submission -> done) is measured on the host clock.
 * Lenses, maps, learned maps and device buffers must stay alive until the
 * ticket completes.  Context: the rendering pipeline of Sec. 4 (Listing 1)
 * queries a path's map for every backward pixel sample and for every forward
 * flare path; such streams of queries are what the server batches.
 */
typedef struct lt_server lt_server;

typedef struct {
    size_t mem_budget_bytes;     /* 0: 1 GiB */
    int32_t n_streams;           /* 0: 4 */
    int32_t fuse_max_requests;   /* requests per fused launch, 1..128 (0: 128) */
    size_t fuse_max_rays;        /* requests up to this size are fused (0: 65536) */
    int32_t inject_fail_every;   /* host-side fault injection for tests: every k-th launch
                                    is not made and its requests fail with LT_ECUDA (0: off) */
    uint32_t batch_window_us;    /* 0: launch what is waiting at once; > 0: hold the oldest
                                    waiting request up to this long while more arrive (until
                                    fuse_max_requests wait), trading latency for fusion */
} lt_server_opts;

enum {
    LT_REQ_TRACE = 0,            /* lt_trace(lens, path_id) */
    LT_REQ_QUERY = 1,            /* lt_query(map, query_mode) */
    LT_REQ_MLP = 2               /* lt_mlp_query(mlp, precision) */
};
#define LT_REQ_HOST_BUFFERS 0x1  /* in, lambda_nm and out are HOST arrays; the server stages them */

typedef struct {
    int32_t kind;                /* LT_REQ_* */
    int32_t flags;               /* LT_REQ_HOST_BUFFERS or 0 (device arrays, 16-byte aligned) */
    const lt_lens* lens;         /* TRACE */
    int32_t path_id;             /* TRACE */
    const lt_map* map;           /* QUERY */
    int32_t query_mode;          /* QUERY: LT_QUERY_TABLE or LT_QUERY_NO_MASK */
    const lt_mlp* mlp;           /* MLP */
    int32_t precision;           /* MLP: LT_MLP_* */
    lt_rays_in in;
    const float* lambda_nm;
    lt_rays_out out;
    size_t n;                    /* < 2^31 */
    uint32_t deadline_us;        /* 0: none */
} lt_request;

typedef struct {
    double queue_us;             /* submission -> launch */
    double latency_us;           /* submission -> completion */
    int32_t fused;               /* requests in the launch that served this one */
} lt_ticket_info;

typedef struct {
    uint64_t submitted, completed, failed, timed_out;
    uint64_t launches, fused_launches, fused_requests, rays;
    size_t bytes_in_flight, peak_bytes_in_flight;
} lt_server_stats;

/* Errors: LT_EINVAL (bad option), LT_ECUDA (stream creation). */
lt_status lt_server_create(const lt_server_opts* opts, lt_server** out);
/* Stops the worker, waits for every launched request, drops unlaunched ones. */
void lt_server_destroy(lt_server* server);
/* Validates and enqueues; *ticket identifies the request.  n = 0 completes at
 * once.  Errors: LT_EINVAL (NULL, unknown kind, bad path id, misaligned or
 * NULL device array, n >= 2^31), LT_ENOMEM (request larger than the budget). */
lt_status lt_submit(lt_server* server, const lt_request* req, uint64_t* ticket);
/* Waits up to timeout_us (0: no wait) for a ticket.  LT_OK: done (the ticket
 * is released); LT_ENOTREADY: not done yet (the ticket stays valid; poll
 * again); the request's own error once it ended unsuccessfully (released):
 * LT_ETIMEOUT (its deadline passed before launch), LT_ECUDA, LT_ENOMEM ...;
 * LT_EINVAL: unknown or already released ticket. */
lt_status lt_poll(lt_server* server, uint64_t ticket, uint32_t timeout_us);
/* lt_poll that also reports the request's timing (info may be NULL). */
lt_status lt_poll_info(lt_server* server, uint64_t ticket, uint32_t timeout_us,
                       lt_ticket_info* info);
lt_status lt_server_stats_get(lt_server* server, lt_server_stats* out);

/* ------------------------------------------------------------------ profiling */

/* Per-kernel device time.  When enabled, each kernel launch of the library
 * is bracketed by two CUDA events recorded on the stream it is launched on
 * (so the times are device times of that kernel alone).  lt_profile_read
 * waits for the recorded events, fills up to `max` entries (one per kernel
 * name, launches and summed milliseconds), sets *n to the number of kernel
 * names seen, and clears the record if `reset` is non-zero.  At most 65,536
 * launches are kept between resets.  While enabled, tracing kernels also
 * count their work (one 64-bit atomic per warp, spread over eight counters
 * per launch so that the counting does not serialise on one address). */
typedef struct {
    char name[48];
    int64_t launches;
    double total_ms;
    int64_t work;        /* tracing kernels: ray-surface interactions evaluated (the image
                            plane counts as one); 0 for other kernels */
} lt_kernel_time;

lt_status lt_profile_enable(int32_t on);
lt_status lt_profile_read(lt_kernel_time* out, int32_t max, int32_t* n, int32_t reset);

/* Thread-local message of the last failed call in this thread ("" if none). */
const char* lt_last_error(void);
/* Library version string. */
const char* lt_version(void);

#ifdef __cplusplus
}
#endif
#endif /* LT_H */
