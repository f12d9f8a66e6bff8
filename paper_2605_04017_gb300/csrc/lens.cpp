// Lens creation, paraxial data, path numbering and error reporting.
//
// The image plane of a lens sits at its paraxial focus for a reference
// wavelength unless the caller fixes it.  The paraxial data come from a
// (y, n*u) marginal-ray trace in FP64: refraction n'u' = n u - y (n' - n) c,
// transfer y' = y + t u'.  With air on both sides EFL = -y_1 / u'_S and the
// back focal distance BFD = -y_S / u'_S.
#include <algorithm>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <new>

#include "lt_internal.h"

namespace lt {

static thread_local std::string g_err;

lt_status fail(lt_status code, const char* fmt, ...)
{
    char buf[512];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof buf, fmt, ap);
    va_end(ap);
    g_err = buf;
    return code;
}

lt_status cuda_fail(cudaError_t e, const char* what)
{
    return fail(LT_ECUDA, "%s: %s", what, cudaGetErrorString(e));
}

void clear_error() { g_err.clear(); }

bool aligned16(const void* p) { return (reinterpret_cast<uintptr_t>(p) & 15u) == 0; }

static double glass_index(const lt_lens* L, int g, double lam_nm)
{
    if (g < 0) return 1.0;
    const lt_glass& G = L->glass[g];
    const double lu = lam_nm * 1e-3, l2 = lu * lu;
    if (G.kind == LT_GLASS_CAUCHY) return G.A + G.B / l2;
    if (G.kind == LT_GLASS_SELLMEIER) {
        double n2 = 1.0;
        for (int i = 0; i < 3; ++i) n2 += G.B3[i] * l2 / (l2 - G.C3[i]);
        return std::sqrt(n2);
    }
    return 1.0;
}

static double medium_index(const lt_lens* L, int m, double lam_nm)
{
    if (m <= 0 || m >= L->S) return 1.0;
    return glass_index(L, L->surf[m - 1].glass_after, lam_nm);
}

int paraxial(const lt_lens* L, double lambda_nm, double* efl, double* bfd)
{
    double y = 1.0, u = 0.0;
    const double y1 = 1.0;
    for (int k = 1; k <= L->S; ++k) {
        if (k > 1) y += (L->zv[k] - L->zv[k - 1]) * u;
        const double n = medium_index(L, k - 1, lambda_nm);
        const double np = medium_index(L, k, lambda_nm);
        const double nu = n * u - y * (np - n) * L->surf[k - 1].curvature;
        u = nu / np;
    }
    if (u == 0.0) return -1;
    *efl = -y1 / u;
    *bfd = -y / u;
    return 0;
}

bool path_ij(int S, int id, int* i, int* j)
{
    if (id == 0) { *i = 0; *j = 0; return true; }
    if (id < 0 || S < 2 || id > S * (S - 1) / 2) return false;
    // row a holds the S - a ghosts (a, a+1..S)
    int a = 1, k = id;
    while (k > S - a) { k -= S - a; ++a; }
    *i = a;
    *j = a + k;
    return true;
}

}  // namespace lt

using namespace lt;

extern "C" {

const char* lt_last_error(void) { return g_err.c_str(); }
const char* lt_version(void) { return "liblt 0.1 (sm_103a)"; }

int32_t lt_path_id(int32_t S, int32_t i, int32_t j)
{
    if (i == 0 && j == 0) return 0;
    if (!(1 <= i && i < j && j <= S)) return -1;
    int32_t id = 0;
    for (int a = 1; a < i; ++a) id += S - a;
    return id + (j - i);
}

lt_status lt_path_ij(int32_t S, int32_t id, int32_t* i, int32_t* j)
{
    int a, b;
    if (!i || !j || !path_ij(S, id, &a, &b)) return fail(LT_EINVAL, "lt_path_ij: bad path id %d for %d surfaces", id, S);
    *i = a;
    *j = b;
    return LT_OK;
}

uint64_t lt_path_code(int32_t S, int32_t i, int32_t j)
{
    if (S < 1) return 0;
    if (i == 0 && j == 0) return S > 63 ? 0 : (1ULL << S);
    if (!(1 <= i && i < j && j <= S)) return 0;
    const int K = S + 2 * (j - i);
    if (K > 63) return 0;
    // interactions are numbered 1..K: reflections at interaction j (surface j
    // going forward) and at interaction 2j - i (surface i coming back)
    return (1ULL << K) | (1ULL << (j - 1)) | (1ULL << (2 * j - i - 1));
}

int32_t lt_lens_n_paths(const lt_lens* L)
{
    if (!L) return 0;
    return 1 + L->S * (L->S - 1) / 2;
}

lt_status lt_lens_paraxial(const lt_lens* L, double lam, double* efl, double* bfd, double* zi)
{
    if (!L) return fail(LT_EINVAL, "lt_lens_paraxial: NULL lens");
    double e, b;
    if (paraxial(L, lam, &e, &b) != 0) return fail(LT_EBADLENS, "lt_lens_paraxial: afocal lens");
    if (efl) *efl = e;
    if (bfd) *bfd = b;
    if (zi) *zi = L->z_image;
    return LT_OK;
}

lt_status lt_create_lens(const lt_prescription* p, lt_lens** out)
{
    clear_error();
    if (!p || !out) return fail(LT_EINVAL, "lt_create_lens: NULL argument");
    *out = nullptr;
    const int S = p->n_surfaces;
    if (S < 1 || S > LT_MAX_SURFACES || !p->surfaces)
        return fail(LT_EINVAL, "lt_create_lens: n_surfaces %d outside 1..%d", S, LT_MAX_SURFACES);
    if (p->n_glasses < 0 || p->n_glasses > LT_MAX_GLASSES || (p->n_glasses > 0 && !p->glasses))
        return fail(LT_EINVAL, "lt_create_lens: n_glasses %d outside 0..%d", p->n_glasses, LT_MAX_GLASSES);
    for (int k = 0; k < S; ++k) {
        const lt_surface& s = p->surfaces[k];
        if (s.glass_after < -1 || s.glass_after >= p->n_glasses)
            return fail(LT_EBADLENS, "surface %d: glass index %d out of range", k + 1, s.glass_after);
        if (!(s.aperture_r > 0.0) || !std::isfinite(s.curvature) ||
            !(std::fabs(s.curvature) * s.aperture_r < 1.0))
            return fail(LT_EBADLENS, "surface %d: aperture must be positive and smaller than |R|", k + 1);
        if (!std::isfinite(s.conic) || !std::isfinite(s.asph[0]) || !std::isfinite(s.asph[1]) ||
            !std::isfinite(s.asph[2]) || !std::isfinite(s.asph[3]) ||
            !(1.0 - (1.0 + s.conic) * s.curvature * s.curvature * s.aperture_r * s.aperture_r > 0.0))
            return fail(LT_EBADLENS, "surface %d: the clear aperture reaches beyond the conic", k + 1);
        if (k + 1 < S && !(s.thickness >= 0.0))
            return fail(LT_EBADLENS, "surface %d: negative thickness", k + 1);
    }
    for (int g = 0; g < p->n_glasses; ++g) {
        const int kd = p->glasses[g].kind;
        if (kd != LT_GLASS_AIR && kd != LT_GLASS_CAUCHY && kd != LT_GLASS_SELLMEIER)
            return fail(LT_EBADLENS, "glass %d: unknown kind %d", g, kd);
    }
    if (p->stop_r > 0.0 && (p->stop_after < 0 || p->stop_after > S))
        return fail(LT_EBADLENS, "stop_after %d outside 0..%d", p->stop_after, S);
    if (!(p->entrance_gap >= 0.0)) return fail(LT_EBADLENS, "negative entrance gap");

    lt_lens* L = new (std::nothrow) lt_lens();
    if (!L) return fail(LT_ENOMEM, "lt_create_lens: out of host memory");
    L->S = S;
    L->n_glass = p->n_glasses;
    std::memcpy(L->surf, p->surfaces, sizeof(lt_surface) * S);
    if (p->n_glasses) std::memcpy(L->glass, p->glasses, sizeof(lt_glass) * p->n_glasses);
    L->surf[S - 1].glass_after = -1;  // the medium behind the lens is air
    L->presc = *p;
    L->presc.surfaces = L->surf;
    L->presc.glasses = L->glass;
    L->zv[0] = 0.0;
    double z = p->entrance_gap;
    for (int k = 1; k <= S; ++k) {
        L->zv[k] = z;
        z += L->surf[k - 1].thickness;
    }
    if (p->image_mode == LT_IMAGE_PARAXIAL) {
        double efl, bfd;
        if (paraxial(L, p->lambda_ref_nm, &efl, &bfd) != 0 || !(bfd > 0.0) ||
            !std::isfinite(bfd)) {
            delete L;
            return fail(LT_EBADLENS, "paraxial image plane: back focal distance must be > 0");
        }
        L->z_image = L->zv[S] + bfd;
    } else if (p->image_mode == LT_IMAGE_ABS) {
        L->z_image = p->image_z;
    } else {
        delete L;
        return fail(LT_EINVAL, "unknown image_mode %d", p->image_mode);
    }

    const double eps = p->edge_eps_mm > 0.0 ? p->edge_eps_mm : 1e-6;
    LensDev& D = L->dev;
    std::memset(&D, 0, sizeof D);
    D.S = S;
    D.med[0] = -1;
    for (int k = 1; k <= S; ++k) D.med[k] = (int8_t)L->surf[k - 1].glass_after;
    D.med[S] = -1;
    for (int g = 0; g < L->n_glass; ++g) {
        const lt_glass& G = L->glass[g];
        D.gkind[g] = (int8_t)G.kind;
        D.gA[g] = (float)G.A;
        D.gB[g] = (float)G.B;
        for (int i = 0; i < 3; ++i) {
            D.gSB[g][i] = (float)G.B3[i];
            D.gSC[g][i] = (float)G.C3[i];
        }
    }
    for (int k = 1; k <= S; ++k) {
        const double a = L->surf[k - 1].aperture_r;
        SurfRec& r = D.s[k];
        r.c = (float)L->surf[k - 1].curvature;
        r.th_before = (float)(L->zv[k] - L->zv[k - 1]);
        r.th_after = k < S ? (float)(L->zv[k + 1] - L->zv[k]) : 0.0f;
        r.ap2 = (float)(a * a);
        r.eps2a = (float)(2.0 * a * eps);
        const int gb = D.med[k - 1], ga = D.med[k];
        r.A_before = gb < 0 ? 1.0f : D.gA[gb];
        r.B_before = gb < 0 ? 0.0f : D.gB[gb];
        r.A_after = ga < 0 ? 1.0f : D.gA[ga];
        r.B_after = ga < 0 ? 0.0f : D.gB[ga];
        r.g_before = (float)gb;
        r.g_after = (float)ga;
        const lt_surface& sf = L->surf[k - 1];
        r.kc = (float)sf.conic;
        r.a4 = (float)sf.asph[0];
        r.a6 = (float)sf.asph[1];
        r.a8 = (float)sf.asph[2];
        r.a10 = (float)sf.asph[3];
    }
    if (p->stop_r > 0.0) {
        const int g = p->stop_after;
        L->z_stop = (g == 0 ? 0.0 : L->zv[g]) + p->stop_offset;
        D.stop_gap = g;
        D.zs_lo = (float)(L->z_stop - L->zv[g]);
        D.zs_hi = (float)(g < S ? L->z_stop - L->zv[g + 1] : 0.0);
        D.a_stop2 = (float)(p->stop_r * p->stop_r);
        D.eps2a_stop = (float)(2.0 * p->stop_r * eps);
    } else {
        D.stop_gap = -1;
        L->z_stop = 0.0;
    }
    D.z_img_rel = (float)(L->z_image - L->zv[S]);
    D.grazing_k = (float)(p->grazing_k > 0.0 ? p->grazing_k : 1e-2);
    *out = L;
    return LT_OK;
}

void lt_destroy_lens(lt_lens* L) { delete L; }

lt_status lt_reverse_lens(const lt_lens* F, double sensor_z, double out_z, lt_lens** out)
{
    clear_error();
    if (!F || !out) return fail(LT_EINVAL, "lt_reverse_lens: NULL argument");
    *out = nullptr;
    const int S = F->S;
    if (!std::isfinite(sensor_z) || !std::isfinite(out_z))
        return fail(LT_EINVAL, "lt_reverse_lens: planes must be finite");
    // the sensor lies behind the last surface's cap, the output plane in front of the first's
    auto sag = [](double c, double a) { return c * a * a / (1.0 + std::sqrt(std::max(0.0, 1.0 - c * c * a * a))); };
    const lt_surface& last = F->surf[S - 1];
    const lt_surface& first = F->surf[0];
    if (!(sensor_z > F->zv[S] + std::max(0.0, sag(last.curvature, last.aperture_r))))
        return fail(LT_EINVAL, "lt_reverse_lens: the sensor plane must lie behind the last surface");
    if (!(out_z <= F->zv[1] + std::min(0.0, sag(first.curvature, first.aperture_r))))
        return fail(LT_EINVAL, "lt_reverse_lens: the output plane must lie in front of the first surface");
    const lt_prescription& P = F->presc;
    if (P.stop_r > 0.0 && !(F->z_stop < sensor_z && F->z_stop >= out_z))
        return fail(LT_EINVAL, "lt_reverse_lens: the stop must lie between the output plane and the sensor");
    lt_surface surf[LT_MAX_SURFACES];
    for (int j = 1; j <= S; ++j) {
        const int k = S + 1 - j;               // forward surface
        const lt_surface& s = F->surf[k - 1];
        surf[j - 1].curvature = -s.curvature;
        surf[j - 1].aperture_r = s.aperture_r;
        surf[j - 1].thickness = k >= 2 ? F->zv[k] - F->zv[k - 1] : 0.0;
        surf[j - 1].glass_after = k >= 2 ? F->surf[k - 2].glass_after : -1;
        // mirroring negates the sag: the polynomial terms change sign, the conic does not
        surf[j - 1].conic = s.conic;
        for (int q = 0; q < 4; ++q) surf[j - 1].asph[q] = -s.asph[q];
    }
    lt_prescription R = P;
    R.surfaces = surf;
    R.glasses = F->glass;
    R.n_glasses = F->n_glass;
    R.entrance_gap = sensor_z - F->zv[S];
    if (P.stop_r > 0.0) {
        const int g = P.stop_after;            // forward gap between vertex g and g + 1
        R.stop_after = S - g;
        R.stop_offset = R.stop_after == 0 ? sensor_z - F->z_stop : F->zv[g + 1] - F->z_stop;
    }
    R.image_mode = LT_IMAGE_ABS;
    R.image_z = sensor_z - out_z;
    return lt_create_lens(&R, out);
}

}  // extern "C"
