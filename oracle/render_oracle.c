/*
 * render_oracle.c -- CPU restatement of the headless renderer (see
 * render_oracle.h).  TEST INFRASTRUCTURE ONLY.  Plain C99, single precision,
 * built without FMA contraction; every expression is evaluated one rounded
 * operation at a time, left to right as written.
 *
 * The paper (Sec. 3) names what is shown -- colormaps of eta, u, v and the
 * velocity magnitude, water rendered with reflection and refraction weighted
 * by the Fresnel equations, a colormap on the terrain and a grid over the
 * surfaces -- but not the colours, the lighting or the camera.  Those are
 * this renderer's own choices, stated at each function.
 */
#include <math.h>
#include <stddef.h>

#include "render_oracle.h"

static const float kN2 = 1.333f;   /* refractive index of water (air: 1) */

/* Colormaps: piecewise linear through 5 control points at t = 0, 1/4, ...,
 * 1 (diverging blue-white-red for signed values, dark-to-bright for the
 * speed, sand-green-brown for the terrain). */
static const float kMaps[3][5][3] = {
    {{0.020f, 0.188f, 0.380f}, {0.263f, 0.576f, 0.765f}, {0.969f, 0.969f, 0.969f},
     {0.957f, 0.647f, 0.510f}, {0.404f, 0.000f, 0.122f}},
    {{0.050f, 0.030f, 0.200f}, {0.150f, 0.250f, 0.550f}, {0.100f, 0.600f, 0.650f},
     {0.550f, 0.850f, 0.350f}, {0.990f, 0.950f, 0.300f}},
    {{0.780f, 0.700f, 0.500f}, {0.600f, 0.650f, 0.380f}, {0.350f, 0.550f, 0.250f},
     {0.450f, 0.480f, 0.300f}, {0.550f, 0.450f, 0.350f}}};

static const float kSkyHorizon[3] = {0.780f, 0.850f, 0.920f};
static const float kSkyZenith[3] = {0.250f, 0.450f, 0.800f};
static const float kWater[3] = {0.020f, 0.150f, 0.200f};

static float clamp01(float x) { return x < 0.0f ? 0.0f : (x > 1.0f ? 1.0f : x); }

void ro_colormap(int which, float t, float rgb[3])
{
    t = clamp01(t);
    float s = t * 4.0f;
    int k = (int)s;
    if (k > 3) k = 3;
    float f = s - (float)k;
    for (int c = 0; c < 3; c++) {
        float a = kMaps[which][k][c], b = kMaps[which][k + 1][c];
        rgb[c] = a + (b - a) * f;
    }
}

/* Fresnel equations for unpolarised light from air (n = 1) into water:
 * R = (rs^2 + rp^2) / 2 with Snell's law for the transmitted angle. */
float ro_fresnel(float cos_i)
{
    cos_i = clamp01(cos_i);
    float sin2_i = 1.0f - cos_i * cos_i;
    float sin2_t = sin2_i / (kN2 * kN2);
    float cos_t = sqrtf(1.0f - sin2_t);
    float rs = (cos_i - kN2 * cos_t) / (cos_i + kN2 * cos_t);
    float rp = (kN2 * cos_i - cos_t) / (kN2 * cos_i + cos_t);
    return (rs * rs + rp * rp) * 0.5f;
}

static void normalize3(float v[3])
{
    float n = sqrtf(v[0] * v[0] + v[1] * v[1] + v[2] * v[2]);
    v[0] = v[0] / n;
    v[1] = v[1] / n;
    v[2] = v[2] / n;
}

static float normalized_value(float v, float lo, float hi) { return (v - lo) / (hi - lo); }

static unsigned char to_byte(float c) { return (unsigned char)(int)(clamp01(c) * 255.0f + 0.5f); }

void ro_render(int nx, int ny, double dx_, double dy_, double ws_, const double *w, const double *P,
               const double *Q, const double *Bbar, const ro_params *p, unsigned char *rgba)
{
    const float dx = (float)dx_, dy = (float)dy_, ws = (float)ws_;
#define AT(a, i, j) ((float)(a)[(size_t)(j) * nx + (i)])
    for (int j = 0; j < ny; j++)
        for (int i = 0; i < nx; i++) {
            const float wc = AT(w, i, j), Bc = AT(Bbar, i, j);
            const float h = wc - Bc;
            const int wet = h > p->dry_h;
            /* neighbours for the gradients, clamped at the edges */
            const int iw = i > 0 ? i - 1 : i, ie = i < nx - 1 ? i + 1 : i;
            const int js = j > 0 ? j - 1 : j, jn = j < ny - 1 ? j + 1 : j;
            const float spanx = (float)(ie - iw) * dx, spany = (float)(jn - js) * dy;
            float rgb[3];
            if (!wet) {
                /* land: terrain colormap with a hillshade from the bed normal */
                float gx = spanx > 0.0f ? (AT(Bbar, ie, j) - AT(Bbar, iw, j)) / spanx : 0.0f;
                float gy = spany > 0.0f ? (AT(Bbar, i, jn) - AT(Bbar, i, js)) / spany : 0.0f;
                float nb[3] = {-(p->exaggeration * gx), -(p->exaggeration * gy), 1.0f};
                normalize3(nb);
                float L[3] = {p->sun[0], p->sun[1], p->sun[2]};
                normalize3(L);
                float d = nb[0] * L[0] + nb[1] * L[1] + nb[2] * L[2];
                float shade = 0.35f + 0.65f * (d > 0.0f ? d : 0.0f);
                ro_colormap(2, normalized_value(Bc, p->zmin, p->zmax), rgb);
                for (int c = 0; c < 3; c++) rgb[c] = rgb[c] * shade;
            } else if (p->mode == RO_FRESNEL) {
                /* water surface normal from eta, with dry neighbours taken level */
                const float ec = wc - ws;
                float eW = AT(w, iw, j) - AT(Bbar, iw, j) > p->dry_h ? AT(w, iw, j) - ws : ec;
                float eE = AT(w, ie, j) - AT(Bbar, ie, j) > p->dry_h ? AT(w, ie, j) - ws : ec;
                float eS = AT(w, i, js) - AT(Bbar, i, js) > p->dry_h ? AT(w, i, js) - ws : ec;
                float eN = AT(w, i, jn) - AT(Bbar, i, jn) > p->dry_h ? AT(w, i, jn) - ws : ec;
                float gx = spanx > 0.0f ? (eE - eW) / spanx : 0.0f;
                float gy = spany > 0.0f ? (eN - eS) / spany : 0.0f;
                float n[3] = {-(p->exaggeration * gx), -(p->exaggeration * gy), 1.0f};
                normalize3(n);
                float I[3] = {p->view[0], p->view[1], p->view[2]};
                normalize3(I);
                float idn = I[0] * n[0] + I[1] * n[1] + I[2] * n[2];
                float R = ro_fresnel(-idn);
                /* reflected ray: sky from the horizon colour up to the zenith colour */
                float rz = I[2] - 2.0f * idn * n[2];
                float tz = clamp01(rz);
                /* refracted ray: the bed colour, weighted down with depth toward the water colour */
                float bed[3];
                ro_colormap(2, normalized_value(Bc, p->zmin, p->zmax), bed);
                float a = 1.0f / (1.0f + p->absorb * h);
                for (int c = 0; c < 3; c++) {
                    float sky = kSkyHorizon[c] + (kSkyZenith[c] - kSkyHorizon[c]) * tz;
                    float refr = kWater[c] + (bed[c] - kWater[c]) * a;
                    rgb[c] = R * sky + (1.0f - R) * refr;
                }
            } else {
                float v;
                int map = 0;
                if (p->mode == RO_ETA) {
                    v = wc - ws;
                } else {
                    float hd = h > p->h_min ? h : p->h_min;
                    float u = AT(P, i, j) / hd, vv = AT(Q, i, j) / hd;
                    if (p->mode == RO_U) v = u;
                    else if (p->mode == RO_V) v = vv;
                    else {
                        v = sqrtf(u * u + vv * vv);
                        map = 1;
                    }
                }
                ro_colormap(map, normalized_value(v, p->vmin, p->vmax), rgb);
            }
            if (p->grid > 0.0f) {
                /* a grid line crosses cell i where floor(x / grid) changes across it */
                int lx = floorf((float)(i + 1) * dx / p->grid) != floorf((float)i * dx / p->grid);
                int ly = floorf((float)(j + 1) * dy / p->grid) != floorf((float)j * dy / p->grid);
                if (lx || ly)
                    for (int c = 0; c < 3; c++) rgb[c] = rgb[c] * 0.6f;
            }
            unsigned char *o = rgba + ((size_t)j * nx + i) * 4;
            o[0] = to_byte(rgb[0]);
            o[1] = to_byte(rgb[1]);
            o[2] = to_byte(rgb[2]);
            o[3] = 255;
        }
#undef AT
}
