/*
 * ORACLE (test infrastructure only): the factorised lens transport map,
 * FP64, one thread.
 *
 * The paper (Sec. 4.2, "Neural Ray Masking", Eq. 11) factorises a path's
 * transport map into a binary valid/occluded mask g(x) and a smooth
 * regressor f(x) used only where g(x) = 1.  The tabulated form computed here
 * (the paper's learned networks are in mlp.py):
 *   - a regular lattice over the 5-D input box (x, y, s_x, s_y, lambda),
 *     s = d_xy / d_z the direction slopes; every node is traced exactly;
 *   - each lattice cell is INVALID (all 32 corners and all fit rays inside
 *     invalid), VALID (all corners and fit rays valid and the largest
 *     position residual of the fit rays against interpolation <= tol), or
 *     BOUNDARY otherwise;
 *   - a query interpolates multilinearly over the 32 corners in a VALID
 *     cell (direction renormalised), returns "no output" in an INVALID cell,
 *     and traces the ray exactly in a BOUNDARY cell or outside the box.
 * The cell index is an integer decided by floating point, so it is taken
 * with the same FP32 operations the GPU uses: u = (v - lo) * inv_step, each
 * step rounded, s = d_x / d_z rounded; the weights are exact FP64.
 */
#include <math.h>
#include <stdlib.h>
#include <string.h>
#include "oracle.h"

int or_trace_one(const or_lens* L, int pi, int pj, double x, double y, double dx, double dy,
                 double dz, double lam_nm, double* out, double* edge, double* kmin);

enum { OR_CELL_INVALID = 0, OR_CELL_VALID = 1, OR_CELL_BOUNDARY = 2 };

/* FP32 lattice constants from the FP64 box: lo, step = (hi-lo)/(res-1), 1/step. */
int or_map_lattice(const int* res, const double* lo, const double* hi, float* lo_f, float* step_f,
                   float* inv_f)
{
    for (int d = 0; d < 5; ++d) {
        if (res[d] < 2 || !(hi[d] > lo[d])) return -1;
        lo_f[d] = (float)lo[d];
        step_f[d] = (float)((hi[d] - lo[d]) / (double)(res[d] - 1));
        inv_f[d] = (float)((double)(res[d] - 1) / (hi[d] - lo[d]));
    }
    return 0;
}

/* FP32 coordinate of node i along dimension d */
static float node_coord(const float* lo_f, const float* step_f, int d, int i)
{
    volatile float prod = (float)i * step_f[d];
    volatile float v = lo_f[d] + prod;
    return v;
}

/* entrance ray of a lattice node, in FP32: direction = normalize(s_x, s_y, 1) */
void or_map_node_ray(const float* lo_f, const float* step_f, const int* idx, float* ray)
{
    float q[5];
    for (int d = 0; d < 5; ++d) q[d] = node_coord(lo_f, step_f, d, idx[d]);
    volatile float a = q[2] * q[2];
    volatile float b = q[3] * q[3];
    volatile float s = a + b;
    volatile float n2 = s + 1.0f;
    volatile float len = sqrtf(n2);
    ray[0] = q[0];
    ray[1] = q[1];
    ray[2] = q[2] / len;
    ray[3] = q[3] / len;
    ray[4] = 1.0f / len;
    ray[5] = q[4];
}

/* 5-D coordinates of a ray in the lattice box, FP32 */
static void ray_coords(float x, float y, float dx, float dy, float dz, float lam, float* v)
{
    volatile float sx = dx / dz;
    volatile float sy = dy / dz;
    v[0] = x; v[1] = y; v[2] = sx; v[3] = sy; v[4] = lam;
}

/* Cell of a ray; returns 1 inside the box, 0 outside (or bad input). */
int or_map_cell_of(const int* res, const float* lo_f, const float* inv_f, const float* ray,
                   int* cell)
{
    float v[5];
    if (!(ray[4] > 0.0f)) return 0;
    ray_coords(ray[0], ray[1], ray[2], ray[3], ray[4], ray[5], v);
    for (int d = 0; d < 5; ++d) {
        volatile float diff = v[d] - lo_f[d];
        volatile float u = diff * inv_f[d];
        if (!(u >= 0.0f && u <= (float)(res[d] - 1))) return 0;
        int c = (int)floorf(u);
        if (c > res[d] - 2) c = res[d] - 2;
        cell[d] = c;
    }
    return 1;
}

static long node_index(const int* res, const int* idx)
{
    long l = 0;
    for (int d = 0; d < 5; ++d) l = l * res[d] + idx[d];
    return l;
}

static long cell_index(const int* res, const int* c)
{
    long l = 0;
    for (int d = 0; d < 5; ++d) l = l * (res[d] - 1) + c[d];
    return l;
}

long or_map_cell_ids(const int* res, const float* lo_f, const float* inv_f, long n, const float* x,
                     const float* y, const float* dx, const float* dy, const float* dz,
                     const float* lam, long* cell_id)
{
    long inside = 0;
    for (long r = 0; r < n; ++r) {
        float ray[6] = {x[r], y[r], dx[r], dy[r], dz[r], lam[r]};
        int c[5];
        if (or_map_cell_of(res, lo_f, inv_f, ray, c)) { cell_id[r] = cell_index(res, c); ++inside; }
        else cell_id[r] = -1;
    }
    return inside;
}

/* Exact FP64 multilinear interpolation over the 32 corners of `cell`. */
static void interpolate(const int* res, const float* lo_f, const float* step_f, const int* cell,
                        const double* corner6 /* 32 x 6, corner bit d = offset along d */,
                        const float* ray, double* out)
{
    double w[5];
    double v[5] = {ray[0], ray[1], 0.0, 0.0, ray[5]};
    /* slopes in FP64 from the FP32 direction */
    v[2] = (double)ray[2] / (double)ray[4];
    v[3] = (double)ray[3] / (double)ray[4];
    for (int d = 0; d < 5; ++d) {
        double a = node_coord(lo_f, step_f, d, cell[d]);
        double b = node_coord(lo_f, step_f, d, cell[d] + 1);
        w[d] = (v[d] - a) / (b - a);
    }
    for (int q = 0; q < 6; ++q) out[q] = 0.0;
    for (int k = 0; k < 32; ++k) {
        double wk = 1.0;
        for (int d = 0; d < 5; ++d) wk *= ((k >> (4 - d)) & 1) ? w[d] : 1.0 - w[d];
        for (int q = 0; q < 6; ++q) out[q] += wk * corner6[k * 6 + q];
    }
    double l = sqrt(out[2] * out[2] + out[3] * out[3] + out[4] * out[4]);
    if (l > 0.0) { out[2] /= l; out[3] /= l; out[4] /= l; }
}

/* corner k of a cell -> node multi-index (bit 4-d of k selects +1 along d) */
static void corner_idx(const int* cell, int k, int* idx)
{
    for (int d = 0; d < 5; ++d) idx[d] = cell[d] + ((k >> (4 - d)) & 1);
}

/* Trace every lattice node.  node6: N x 6, node_valid: N.  Returns valid nodes. */
long or_map_trace_nodes(const or_lens* L, int pi, int pj, const int* res, const float* lo_f,
                        const float* step_f, double* node6, unsigned char* node_valid)
{
    long N = 1;
    for (int d = 0; d < 5; ++d) N *= res[d];
    long nv = 0;
    int idx[5];
    for (long l = 0; l < N; ++l) {
        long t = l;
        for (int d = 4; d >= 0; --d) { idx[d] = (int)(t % res[d]); t /= res[d]; }
        float ray[6];
        or_map_node_ray(lo_f, step_f, idx, ray);
        double e, km;
        int v = or_trace_one(L, pi, pj, ray[0], ray[1], ray[2], ray[3], ray[4], ray[5],
                             node6 + 6 * l, &e, &km);
        node_valid[l] = (unsigned char)(v == 1);
        nv += (v == 1);
    }
    return nv;
}

/*
 * Classify one cell from its 32 traced corners and the fit rays inside it
 * (given by index list).  Also returns the largest position residual (mm)
 * of valid fit rays against interpolation when all corners are valid.
 */
int or_map_classify_cell(const or_lens* L, int pi, int pj, const int* res, const float* lo_f,
                         const float* step_f, const int* cell, const double* corner6,
                         const unsigned char* corner_valid, long nfit, const float* x,
                         const float* y, const float* dx, const float* dy, const float* dz,
                         const float* lam, double tol, double* maxres, long* nvalid,
                         long* ninvalid)
{
    int allv = 1, alli = 1;
    for (int k = 0; k < 32; ++k) {
        if (corner_valid[k]) alli = 0; else allv = 0;
    }
    long nv = 0, ni = 0;
    double mr = 0.0;
    for (long r = 0; r < nfit; ++r) {
        double out[6], e, km;
        int v = or_trace_one(L, pi, pj, x[r], y[r], dx[r], dy[r], dz[r], lam[r], out, &e, &km);
        if (v == 1) {
            ++nv;
            if (allv) {
                float ray[6] = {x[r], y[r], dx[r], dy[r], dz[r], lam[r]};
                double ip[6];
                interpolate(res, lo_f, step_f, cell, corner6, ray, ip);
                double res_mm = hypot(ip[0] - out[0], ip[1] - out[1]);
                if (res_mm > mr) mr = res_mm;
            }
        } else {
            ++ni;
        }
    }
    if (maxres) *maxres = mr;
    if (nvalid) *nvalid = nv;
    if (ninvalid) *ninvalid = ni;
    if (alli && nv == 0) return OR_CELL_INVALID;
    if (allv && ni == 0 && mr <= tol) return OR_CELL_VALID;
    return OR_CELL_BOUNDARY;
}

/*
 * Whole-map build: trace nodes, then classify every cell with the fit rays
 * (fit_cell[r] = cell id from or_map_cell_ids, -1 outside).  cell_class has
 * prod(res-1) entries.  Returns the number of VALID cells.
 */
long or_map_build(const or_lens* L, int pi, int pj, const int* res, const float* lo_f,
                  const float* step_f, const float* inv_f, long nfit, const float* x,
                  const float* y, const float* dx, const float* dy, const float* dz,
                  const float* lam, double tol, double* node6, unsigned char* node_valid,
                  unsigned char* cell_class, double* cell_maxres)
{
    or_map_trace_nodes(L, pi, pj, res, lo_f, step_f, node6, node_valid);
    long NC = 1;
    for (int d = 0; d < 5; ++d) NC *= (res[d] - 1);
    long* cid = (long*)malloc(sizeof(long) * (nfit > 0 ? nfit : 1));
    or_map_cell_ids(res, lo_f, inv_f, nfit, x, y, dx, dy, dz, lam, cid);
    /* bucket the fit rays by cell (counting sort) */
    long* start = (long*)calloc(NC + 1, sizeof(long));
    long* order = (long*)malloc(sizeof(long) * (nfit > 0 ? nfit : 1));
    for (long r = 0; r < nfit; ++r) if (cid[r] >= 0) start[cid[r] + 1]++;
    for (long c = 0; c < NC; ++c) start[c + 1] += start[c];
    long* fill = (long*)malloc(sizeof(long) * (NC > 0 ? NC : 1));
    for (long c = 0; c < NC; ++c) fill[c] = start[c];
    for (long r = 0; r < nfit; ++r) if (cid[r] >= 0) order[fill[cid[r]]++] = r;
    free(fill);

    long nvalid_cells = 0;
    float* bx = (float*)malloc(sizeof(float) * 6 * (nfit > 0 ? nfit : 1));
    int cell[5];
    for (long c = 0; c < NC; ++c) {
        long t = c;
        for (int d = 4; d >= 0; --d) { cell[d] = (int)(t % (res[d] - 1)); t /= (res[d] - 1); }
        double corner6[32 * 6];
        unsigned char cv[32];
        for (int k = 0; k < 32; ++k) {
            int idx[5];
            corner_idx(cell, k, idx);
            long l = node_index(res, idx);
            memcpy(corner6 + 6 * k, node6 + 6 * l, sizeof(double) * 6);
            cv[k] = node_valid[l];
        }
        long m = start[c + 1] - start[c];
        float *fx = bx, *fy = bx + m, *fdx = bx + 2 * m, *fdy = bx + 3 * m, *fdz = bx + 4 * m,
              *fl = bx + 5 * m;
        for (long q = 0; q < m; ++q) {
            long r = order[start[c] + q];
            fx[q] = x[r]; fy[q] = y[r]; fdx[q] = dx[r]; fdy[q] = dy[r]; fdz[q] = dz[r];
            fl[q] = lam[r];
        }
        double mr;
        int cls = or_map_classify_cell(L, pi, pj, res, lo_f, step_f, cell, corner6, cv, m, fx, fy,
                                       fdx, fdy, fdz, fl, tol, &mr, NULL, NULL);
        cell_class[c] = (unsigned char)cls;
        if (cell_maxres) cell_maxres[c] = mr;
        nvalid_cells += (cls == OR_CELL_VALID);
    }
    free(bx); free(order); free(start); free(cid);
    return nvalid_cells;
}

/*
 * Query a built map.  out6: n x 6; flags[r]: bit0 valid, bit3 bad input,
 * bit4 answered by the exact tracer, bit5 outside the lattice box.
 */
long or_map_query(const or_lens* L, int pi, int pj, const int* res, const float* lo_f,
                  const float* step_f, const float* inv_f, const double* node6,
                  const unsigned char* node_valid, const unsigned char* cell_class, long n,
                  const float* x, const float* y, const float* dx, const float* dy,
                  const float* dz, const float* lam, double* out6, unsigned char* flags)
{
    long nv = 0;
    for (long r = 0; r < n; ++r) {
        float ray[6] = {x[r], y[r], dx[r], dy[r], dz[r], lam[r]};
        double* o = out6 + 6 * r;
        for (int q = 0; q < 6; ++q) o[q] = 0.0;
        unsigned char f = 0;
        int cell[5];
        int inside = or_map_cell_of(res, lo_f, inv_f, ray, cell);
        int cls = inside ? cell_class[cell_index(res, cell)] : OR_CELL_BOUNDARY;
        if (!inside) f |= 32;
        if (cls == OR_CELL_VALID) {
            double corner6[32 * 6];
            for (int k = 0; k < 32; ++k) {
                int idx[5];
                corner_idx(cell, k, idx);
                memcpy(corner6 + 6 * k, node6 + 6 * node_index(res, idx), sizeof(double) * 6);
            }
            interpolate(res, lo_f, step_f, cell, corner6, ray, o);
            f |= 1;
        } else if (cls == OR_CELL_BOUNDARY) {
            double e, km;
            int v = or_trace_one(L, pi, pj, ray[0], ray[1], ray[2], ray[3], ray[4], ray[5], o, &e,
                                 &km);
            f |= 16;
            if (v == 1) f |= 1;
            if (v < 0) f |= 8;
        }
        flags[r] = f;
        nv += (f & 1);
    }
    return nv;
}

/* One query answered from scratch: the cell's corners are traced here, and its
 * class is decided from them plus the given fit rays of that cell. */
int or_map_query_one(const or_lens* L, int pi, int pj, const int* res, const float* lo_f,
                     const float* step_f, const float* inv_f, const float* ray, long nfit,
                     const float* x, const float* y, const float* dx, const float* dy,
                     const float* dz, const float* lam, double tol, double* out, int* cls_out)
{
    int cell[5];
    for (int q = 0; q < 6; ++q) out[q] = 0.0;
    double e, km;
    if (!or_map_cell_of(res, lo_f, inv_f, ray, cell)) {
        *cls_out = -1;
        int v = or_trace_one(L, pi, pj, ray[0], ray[1], ray[2], ray[3], ray[4], ray[5], out, &e, &km);
        return v == 1;
    }
    double corner6[32 * 6];
    unsigned char cv[32];
    for (int k = 0; k < 32; ++k) {
        int idx[5];
        float nr[6];
        corner_idx(cell, k, idx);
        or_map_node_ray(lo_f, step_f, idx, nr);
        int v = or_trace_one(L, pi, pj, nr[0], nr[1], nr[2], nr[3], nr[4], nr[5], corner6 + 6 * k,
                             &e, &km);
        cv[k] = (unsigned char)(v == 1);
    }
    int cls = or_map_classify_cell(L, pi, pj, res, lo_f, step_f, cell, corner6, cv, nfit, x, y, dx,
                                   dy, dz, lam, tol, NULL, NULL, NULL);
    *cls_out = cls;
    if (cls == OR_CELL_VALID) { interpolate(res, lo_f, step_f, cell, corner6, ray, out); return 1; }
    if (cls == OR_CELL_INVALID) return 0;
    int v = or_trace_one(L, pi, pj, ray[0], ray[1], ray[2], ray[3], ray[4], ray[5], out, &e, &km);
    return v == 1;
}

/* Interpolate an arbitrary corner table (for the affine-field pin). */
void or_map_interpolate(const int* res, const float* lo_f, const float* step_f, const float* inv_f,
                        const double* corner6, const float* ray, double* out, int* cell)
{
    or_map_cell_of(res, lo_f, inv_f, ray, cell);
    interpolate(res, lo_f, step_f, cell, corner6, ray, out);
}

/* All lattice node entrance rays as SoA arrays (node order of the table). */
void or_map_node_rays(const int* res, const float* lo_f, const float* step_f, float* x, float* y,
                      float* dx, float* dy, float* dz, float* lam)
{
    long N = 1;
    for (int d = 0; d < 5; ++d) N *= res[d];
    int idx[5];
    for (long l = 0; l < N; ++l) {
        long t = l;
        for (int d = 4; d >= 0; --d) { idx[d] = (int)(t % res[d]); t /= res[d]; }
        float ray[6];
        or_map_node_ray(lo_f, step_f, idx, ray);
        x[l] = ray[0]; y[l] = ray[1]; dx[l] = ray[2]; dy[l] = ray[3]; dz[l] = ray[4]; lam[l] = ray[5];
    }
}
