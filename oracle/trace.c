/*
 * ORACLE (test infrastructure only): sequential FP64 lens tracer.
 *
 * What it computes, and where the paper defines it:
 *   - ray state y = [x, omega, I, lambda]                    (Sec. 3, Eq. 2)
 *   - light path P = (L_1..L_K), L in {T, R}, surfaces
 *     sigma_1..sigma_{K+1}, the last one the output plane    (Sec. 3, Eq. 3-4)
 *   - one interaction S_{L,sigma} = closest hit p_sigma, new
 *     direction d_{L,sigma}, Fresnel factor f_{L,sigma}       (Sec. 3, Eq. 5)
 *   - the path operator as their composition                (Sec. 3, Eq. 6-7)
 *   - valid iff the last surface reached is the output plane (Sec. 3)
 *   - apertures / housing absorb rays                        (Sec. 1, Sec. 4.2)
 *   - two-bounce ghost paths only                            (Sec. 4.2)
 * The paper gives no formulas for p, d or f; the readings used are the
 * textbook ones: sphere/plane hit in vertex-local form with the stable
 * quadratic root, vector Snell's law with total internal reflection, mirror
 * reflection, and unpolarised Fresnel reflectance R = (Rs + Rp)/2 with
 * T = 1 - R.  Dispersion: Cauchy n = A + B/lam^2 or 3-term Sellmeier.
 * Paraxial image plane: the ABCD (y, n*u) matrix product of the system.
 */
#include <math.h>
#include <string.h>
#include "oracle.h"

int or_lens_sizeof(void) { return (int)sizeof(or_lens); }

/* read-back of derived lens quantities: 0 image-plane z, 1 stop z, 2 stop radius,
 * 3 stop gap, 100+k vertex z of surface k */
double or_lens_get(const or_lens* L, int what)
{
    if (what == 0) return L->z_image;
    if (what == 1) return L->z_stop;
    if (what == 2) return L->a_stop;
    if (what == 3) return (double)L->stop_gap;
    if (what >= 101 && what <= 100 + L->S) return L->zv[what - 100];
    return NAN;
}

/* refractive index of medium m at wavelength lam_nm */
double or_index(const or_lens* L, int m, double lam_nm)
{
    int g = L->med[m];
    if (g < 0) return 1.0;
    double lu = lam_nm * 1e-3;
    double l2 = lu * lu;
    if (L->gkind[g] == OR_CAUCHY) return L->gA[g] + L->gB[g] / l2;
    if (L->gkind[g] == OR_SELLMEIER) {
        double n2 = 1.0;
        for (int i = 0; i < 3; ++i) n2 += L->gSB[g][i] * l2 / (l2 - L->gSC[g][i]);
        return sqrt(n2);
    }
    return 1.0;
}

/*
 * Paraxial system matrix from surface 1 to surface S acting on (y, n*u):
 * refraction by power phi = (n2 - n1) c is [[1, 0], [-phi, 1]], transfer by
 * thickness t in index n is [[1, t/n], [0, 1]].  With air on both sides the
 * effective focal length is -1/C and the back focal distance -A/C.
 */
int or_paraxial(const or_lens* L, double lam_nm, double* efl, double* bfd)
{
    double A = 1, B = 0, C = 0, D = 1;
    for (int k = 1; k <= L->S; ++k) {
        if (k > 1) {
            double t = L->zv[k] - L->zv[k - 1];
            double n = or_index(L, k - 1, lam_nm);
            double tn = t / n;
            /* [[1, tn], [0, 1]] * M */
            A = A + tn * C;
            B = B + tn * D;
        }
        double phi = (or_index(L, k, lam_nm) - or_index(L, k - 1, lam_nm)) * L->c[k];
        /* [[1, 0], [-phi, 1]] * M */
        C = C - phi * A;
        D = D - phi * B;
    }
    if (C == 0.0) return -1;
    *efl = -1.0 / C;
    *bfd = -A / C;
    return 0;
}

/*
 * Build the oracle's lens from a flat prescription.
 *   curv[k], thick[k], ap[k], glass_after[k] for k = 0..S-1 (surface k+1)
 *   gkind[g], gcoef[g*8 + (A, B, B1, B2, B3, C1, C2, C3)]
 * Returns 0, or -1 for a bad prescription / non-positive back focal distance.
 */
int or_lens_init(or_lens* L, int S, const double* curv, const double* thick, const double* ap,
                 const int* glass_after, int n_glass, const int* gkind, const double* gcoef,
                 double entrance_gap, int stop_after, double stop_offset, double stop_r,
                 int image_mode, double image_z, double lambda_ref_nm)
{
    memset(L, 0, sizeof(*L));
    if (S < 1 || S > OR_MAXS || n_glass < 0 || n_glass > OR_MAXG) return -1;
    L->S = S;
    L->n_glass = n_glass;
    for (int g = 0; g < n_glass; ++g) {
        L->gkind[g] = gkind[g];
        L->gA[g] = gcoef[g * 8 + 0];
        L->gB[g] = gcoef[g * 8 + 1];
        for (int i = 0; i < 3; ++i) {
            L->gSB[g][i] = gcoef[g * 8 + 2 + i];
            L->gSC[g][i] = gcoef[g * 8 + 5 + i];
        }
    }
    L->med[0] = -1;
    double z = entrance_gap;
    for (int k = 1; k <= S; ++k) {
        L->zv[k] = z;
        L->c[k] = curv[k - 1];
        L->ap[k] = ap[k - 1];
        L->med[k] = glass_after[k - 1];
        if (L->med[k] >= n_glass) return -1;
        z += thick[k - 1];
    }
    L->med[S] = -1;        /* the medium after the last surface is air */
    if (stop_r > 0.0 && stop_after >= 0 && stop_after <= S) {
        L->stop_gap = stop_after;
        L->z_stop = (stop_after == 0 ? 0.0 : L->zv[stop_after]) + stop_offset;
        L->a_stop = stop_r;
    } else {
        L->stop_gap = -1;
    }
    if (image_mode == 0) {
        double efl, bfd;
        if (or_paraxial(L, lambda_ref_nm, &efl, &bfd) != 0) return -1;
        if (!(bfd > 0.0)) return -1;
        L->z_image = L->zv[S] + bfd;
    } else {
        L->z_image = image_z;
    }
    return 0;
}

/*
 * Make surface k (1..S) an even asphere (the circularly symmetric surfaces
 * the paper's model admits, Sec. 4.1): sag
 *   z(r) = c r^2 / (1 + sqrt(1 - (1 + kappa) c^2 r^2)) + A4 r^4 + A6 r^6 + A8 r^8 + A10 r^10
 * in the vertex frame.  on = 0 restores the sphere.  Returns 0, or -1 for a
 * bad k or a clear aperture beyond the conic's domain.
 */
int or_lens_set_asphere(or_lens* L, int k, int on, double kappa, const double* a)
{
    if (k < 1 || k > L->S) return -1;
    L->asph[k] = on;
    L->conic[k] = kappa;
    for (int i = 0; i < 4; ++i) L->a4[k][i] = a ? a[i] : 0.0;
    if (on && 1.0 - (1.0 + kappa) * L->c[k] * L->c[k] * L->ap[k] * L->ap[k] < 0.0) return -1;
    return 0;
}

/* sag of an even asphere and its derivative with respect to s = r^2; -1 if
 * s lies beyond the conic's domain */
static int asph_sag(const or_lens* L, int k, double s, double* z, double* dz_ds)
{
    double c = L->c[k];
    double q2 = 1.0 - (1.0 + L->conic[k]) * c * c * s;
    if (q2 < 0.0) return -1;
    double q = sqrt(q2);
    const double* A = L->a4[k];
    double poly = s * s * (A[0] + s * (A[1] + s * (A[2] + s * A[3])));
    double dpoly = s * (2.0 * A[0] + s * (3.0 * A[1] + s * (4.0 * A[2] + s * 5.0 * A[3])));
    *z = c * s / (1.0 + q) + poly;
    /* d/ds [c s / (1 + q)] = c / (2 q) */
    *dz_ds = (q > 0.0 ? c / (2.0 * q) : INFINITY) + dpoly;
    return 0;
}

/*
 * Hit of an even asphere by the ray o + t d (vertex frame): Newton's method
 * on g(t) = o_z + t d_z - z(s(t)), s(t) = |(o + t d)_xy|^2, from t0 (the base
 * sphere's near-cap root, or the vertex plane's).  Returns 0 with *t, or -1
 * (no root the iteration reaches, or a point beyond the conic's domain).
 */
static int asph_hit(const or_lens* L, int k, const double* o, const double* d, double t0, double* t)
{
    double tt = t0;
    for (int it = 0; it < 60; ++it) {
        double px = o[0] + tt * d[0], py = o[1] + tt * d[1];
        double z, zs;
        if (asph_sag(L, k, px * px + py * py, &z, &zs) != 0) return -1;
        double g = o[2] + tt * d[2] - z;
        double gp = d[2] - zs * 2.0 * (px * d[0] + py * d[1]);
        if (gp == 0.0 || !isfinite(gp)) return -1;
        double step = g / gp;
        tt -= step;
        if (fabs(step) <= 1e-14 * (1.0 + fabs(tt))) { *t = tt; return 0; }
    }
    return -1;
}

/*
 * Unpolarised Fresnel reflectance at an interface n1 -> n2 for an incidence
 * cosine cos_i > 0.  Returns 1 for total internal reflection (Rs = Rp = 1).
 */
int or_fresnel(double n1, double n2, double cos_i, double* Rs, double* Rp, double* cos_t)
{
    double eta = n1 / n2;
    double k = 1.0 - eta * eta * (1.0 - cos_i * cos_i);
    if (k < 0.0) {
        *Rs = 1.0; *Rp = 1.0; *cos_t = 0.0;
        return 1;
    }
    double ct = sqrt(k);
    double rs = (n1 * cos_i - n2 * ct) / (n1 * cos_i + n2 * ct);
    double rp = (n1 * ct - n2 * cos_i) / (n1 * ct + n2 * cos_i);
    *Rs = rs * rs;
    *Rp = rp * rp;
    *cos_t = ct;
    return 0;
}

/*
 * Interaction sequence of a path (Sec. 3 Eq. 3; Sec. 4.2: at most two
 * reflections).  (i, j) = (0, 0) is the transmission path 1..S.  A ghost
 * (i, j), 1 <= i < j <= S, goes forward 1..j reflecting at j, backward
 * j-1..i reflecting at i, then forward i+1..S.  Fills surf/type/dir
 * (dir +1 forward, -1 backward) and returns K, or -1 for a bad (i, j).
 */
int or_path_sequence(int S, int i, int j, int* surf, int* type, int* dir)
{
    int K = 0;
    if (i == 0 && j == 0) {
        for (int s = 1; s <= S; ++s) { surf[K] = s; type[K] = OR_T; dir[K] = +1; ++K; }
        return K;
    }
    if (!(1 <= i && i < j && j <= S)) return -1;
    for (int s = 1; s <= j; ++s) { surf[K] = s; type[K] = (s == j) ? OR_R : OR_T; dir[K] = +1; ++K; }
    for (int s = j - 1; s >= i; --s) { surf[K] = s; type[K] = (s == i) ? OR_R : OR_T; dir[K] = -1; ++K; }
    for (int s = i + 1; s <= S; ++s) { surf[K] = s; type[K] = OR_T; dir[K] = +1; ++K; }
    return K;
}

/* Paper-style binary path code: bit (k-1) is 1 when interaction k reflects
 * (least significant bit = first interaction), plus a leading 1 at bit K. */
unsigned long long or_path_code(int S, int i, int j)
{
    int surf[3 * OR_MAXS + 4], type[3 * OR_MAXS + 4], dir[3 * OR_MAXS + 4];
    int K = or_path_sequence(S, i, j, surf, type, dir);
    if (K < 0 || K > 63) return 0;
    unsigned long long code = 1ULL << K;
    for (int k = 0; k < K; ++k)
        if (type[k] == OR_R) code |= 1ULL << k;
    return code;
}

/* Path id -> (i, j): 0 is the transmission path, 1.. enumerate i < j lexicographically. */
int or_path_ij(int S, int id, int* i, int* j)
{
    if (id == 0) { *i = 0; *j = 0; return 0; }
    int k = 0;
    for (int a = 1; a <= S; ++a)
        for (int b = a + 1; b <= S; ++b)
            if (++k == id) { *i = a; *j = b; return 0; }
    return -1;
}

/* edge distance of a point at squared radius r2 to a circle of radius a */
static double edge_distance(double r2, double a) { return fabs(sqrt(r2) - a); }

/*
 * Trace one ray along path (i, j).  Inputs: entrance point (x, y, 0),
 * direction (dx, dy, dz) (normalised here), wavelength.  Outputs: out[0..5]
 * = exit x, y at the image plane, exit direction, throughput I (I_in = 1).
 * Returns 1 if valid, 0 if absorbed/blocked, -1 for a bad input.
 * *edge: smallest |r - a| over the aperture and stop tests made;
 * *kmin: smallest |k| = |1 - eta^2 sin^2 i| over the interactions made.
 */
static int trace_impl(const or_lens* L, int pi, int pj, double x, double y, double dx,
                      double dy, double dz, double lam_nm, double* out, double* edge,
                      double* kmin, double* states, int* nstates);

int or_trace_one(const or_lens* L, int pi, int pj, double x, double y, double dx, double dy,
                 double dz, double lam_nm, double* out, double* edge, double* kmin)
{
    return trace_impl(L, pi, pj, x, y, dx, dy, dz, lam_nm, out, edge, kmin, NULL, NULL);
}

/* Same, recording the state after every interaction and at the output plane:
 * states[7*m + (x, y, z, dx, dy, dz, I)], m = 0..; *nstates = records made. */
int or_trace_states(const or_lens* L, int pi, int pj, double x, double y, double dx, double dy,
                    double dz, double lam_nm, double* out, double* states, int* nstates)
{
    double e, k;
    return trace_impl(L, pi, pj, x, y, dx, dy, dz, lam_nm, out, &e, &k, states, nstates);
}

static void record(double* states, int* nstates, const double* p, const double* d, double I)
{
    if (!states) return;
    double* s = states + 7 * (*nstates);
    s[0] = p[0]; s[1] = p[1]; s[2] = p[2]; s[3] = d[0]; s[4] = d[1]; s[5] = d[2]; s[6] = I;
    ++*nstates;
}

static int trace_impl(const or_lens* L, int pi, int pj, double x, double y, double dx,
                      double dy, double dz, double lam_nm, double* out, double* edge,
                      double* kmin, double* states, int* nstates)
{
    int surf[3 * OR_MAXS + 4], type[3 * OR_MAXS + 4], dir[3 * OR_MAXS + 4];
    for (int q = 0; q < 6; ++q) out[q] = 0.0;
    *edge = INFINITY;
    *kmin = INFINITY;
    if (nstates) *nstates = 0;
    if (!(isfinite(x) && isfinite(y) && isfinite(dx) && isfinite(dy) && isfinite(dz) &&
          isfinite(lam_nm)) || !(dz > 0.0) || !(lam_nm > 0.0))
        return -1;
    int K = or_path_sequence(L->S, pi, pj, surf, type, dir);
    if (K < 0) return -1;

    double nrm = sqrt(dx * dx + dy * dy + dz * dz);
    double d[3] = {dx / nrm, dy / nrm, dz / nrm};
    double p[3] = {x, y, 0.0};
    double I = 1.0;
    double nmed[OR_MAXS + 2];
    for (int m = 0; m <= L->S; ++m) nmed[m] = or_index(L, m, lam_nm);

    int gap = 0;   /* the ray starts in gap 0, between the entrance plane and surface 1 */
    for (int k = 0; k <= K; ++k) {
        /* the segment from p to the next surface lies in gap `gap` */
        double t;
        double hit[3];
        if (k < K) {
            int s = surf[k];
            double c = L->c[s];
            double o[3] = {p[0], p[1], p[2] - L->zv[s]};
            double b = c * (o[0] * d[0] + o[1] * d[1] + o[2] * d[2]) - d[2];
            double C = c * (o[0] * o[0] + o[1] * o[1] + o[2] * o[2]) - 2.0 * o[2];
            double disc = b * b - c * C;
            if (L->asph[s]) {
                /* start from the base sphere's near cap, or the vertex plane */
                double t0 = -o[2] / d[2];
                if (disc >= 0.0) {
                    double q0 = -b - copysign(sqrt(disc), b);
                    if (q0 != 0.0) t0 = C / q0;
                }
                if (asph_hit(L, s, o, d, t0, &t) != 0) return 0;
                if (!(t >= 0.0)) return 0;
            } else {
                if (disc < 0.0) return 0;
                double q = -b - copysign(sqrt(disc), b);
                if (q == 0.0) return 0;
                t = C / q;
                /* t = 0 is a hit at the start point (the singlet's entrance plane
                 * touches its front vertex); only a surface behind the ray misses */
                if (!(t >= 0.0)) return 0;
            }
        } else {
            if (!(d[2] > 0.0)) return 0;
            t = (L->z_image - p[2]) / d[2];
        }
        for (int a = 0; a < 3; ++a) hit[a] = p[a] + t * d[a];

        /* aperture stop: a plane disc tested on the segment crossing its gap */
        if (gap == L->stop_gap) {
            double ts = (L->z_stop - p[2]) / d[2];
            if (ts >= 0.0 && ts <= t) {
                double sx = p[0] + ts * d[0], sy = p[1] + ts * d[1];
                double r2 = sx * sx + sy * sy;
                double e = edge_distance(r2, L->a_stop);
                if (e < *edge) *edge = e;
                if (r2 > L->a_stop * L->a_stop) return 0;
            }
        }
        p[0] = hit[0]; p[1] = hit[1]; p[2] = hit[2];
        if (k == K) { record(states, nstates, p, d, I); break; }

        int s = surf[k];
        /* clear aperture of the surface: a closed disc */
        double r2 = p[0] * p[0] + p[1] * p[1];
        double e = edge_distance(r2, L->ap[s]);
        if (e < *edge) *edge = e;
        if (r2 > L->ap[s] * L->ap[s]) return 0;

        /* unit normal at the hit, facing the incoming ray: of c|p|^2 - 2 p_z = 0
         * for a sphere, of p_z - z(s) = 0 (gradient (-2x z'(s), -2y z'(s), 1))
         * for an asphere */
        double c = L->c[s];
        double nv[3] = {c * p[0], c * p[1], c * (p[2] - L->zv[s]) - 1.0};
        if (L->asph[s]) {
            double z, zs;
            if (asph_sag(L, s, r2, &z, &zs) != 0) return 0;
            nv[0] = -2.0 * p[0] * zs;
            nv[1] = -2.0 * p[1] * zs;
            nv[2] = 1.0;
        }
        double nn = sqrt(nv[0] * nv[0] + nv[1] * nv[1] + nv[2] * nv[2]);
        for (int a = 0; a < 3; ++a) nv[a] /= nn;
        double dn = nv[0] * d[0] + nv[1] * d[1] + nv[2] * d[2];
        if (dn > 0.0) { for (int a = 0; a < 3; ++a) nv[a] = -nv[a]; dn = -dn; }
        double cos_i = -dn;

        double n1, n2;
        if (dir[k] > 0) { n1 = nmed[s - 1]; n2 = nmed[s]; }
        else            { n1 = nmed[s];     n2 = nmed[s - 1]; }
        double eta = n1 / n2;
        double kk = 1.0 - eta * eta * (1.0 - cos_i * cos_i);
        if (fabs(kk) < *kmin) *kmin = fabs(kk);
        double Rs, Rp, ct;
        int tir = or_fresnel(n1, n2, cos_i, &Rs, &Rp, &ct);
        double R = 0.5 * (Rs + Rp);
        if (type[k] == OR_T) {
            if (tir) return 0;
            double nd[3];
            for (int a = 0; a < 3; ++a) nd[a] = eta * d[a] + (eta * cos_i - ct) * nv[a];
            double l = sqrt(nd[0] * nd[0] + nd[1] * nd[1] + nd[2] * nd[2]);
            for (int a = 0; a < 3; ++a) d[a] = nd[a] / l;
            I *= 1.0 - R;
        } else {
            for (int a = 0; a < 3; ++a) d[a] = d[a] + 2.0 * cos_i * nv[a];
            double l = sqrt(d[0] * d[0] + d[1] * d[1] + d[2] * d[2]);
            for (int a = 0; a < 3; ++a) d[a] /= l;
            I *= R;
        }
        record(states, nstates, p, d, I);
        /* the next segment: forward from s lies in gap s, backward from s in gap s-1 */
        int ndir = (k + 1 < K) ? dir[k + 1] : +1;
        gap = (ndir > 0) ? s : s - 1;
    }
    out[0] = p[0]; out[1] = p[1];
    out[2] = d[0]; out[3] = d[1]; out[4] = d[2];
    out[5] = I;
    return 1;
}

/*
 * Batch form.  Inputs are the FP32 ray arrays both sides receive; they are
 * widened to FP64 exactly.  out6 is n x 6 row-major; valid[n] is 1/0 (bad
 * inputs give 0 and bit 3 set).  edge/kmin may be NULL.  Returns the number
 * of valid rays.
 */
long or_trace(const or_lens* L, int pi, int pj, long n, const float* x, const float* y,
              const float* dx, const float* dy, const float* dz, const float* lam,
              double* out6, unsigned char* valid, double* edge, double* kmin)
{
    long nv = 0;
    for (long r = 0; r < n; ++r) {
        double e, km;
        int v = or_trace_one(L, pi, pj, x[r], y[r], dx[r], dy[r], dz[r], lam[r], out6 + 6 * r,
                             &e, &km);
        valid[r] = (unsigned char)(v == 1 ? 1 : (v < 0 ? 8 : 0));
        if (edge) edge[r] = e;
        if (kmin) kmin[r] = km;
        nv += (v == 1);
    }
    return nv;
}
