// Headless rendering of the state into an RGBA8 image: the visualisation
// options of Sec. 3 (colormaps of eta, u, v and the velocity magnitude, water
// shaded by the Fresnel equations, a colormap on the terrain, a grid over the
// surfaces), without any graphics API.
//
// The shading is single precision with every operation rounded on its own
// (the _rn intrinsics: no contraction into fused multiply-adds, IEEE
// division and square root whatever the build's fast-math flags), and no
// transcendental functions, so the bytes are reproducible by any correct
// implementation of the same sequence of operations.  The colours, the
// lighting and the camera are this renderer's choices (the paper names only
// what is shown).
#include "celeris_internal.cuh"

namespace cel {
namespace {

__device__ __forceinline__ float ad(float a, float b) { return __fadd_rn(a, b); }
__device__ __forceinline__ float sb(float a, float b) { return __fsub_rn(a, b); }
__device__ __forceinline__ float ml(float a, float b) { return __fmul_rn(a, b); }
__device__ __forceinline__ float dv(float a, float b) { return __fdiv_rn(a, b); }
__device__ __forceinline__ float sq(float a) { return __fsqrt_rn(a); }
__device__ __forceinline__ float clamp01(float x) { return x < 0.0f ? 0.0f : (x > 1.0f ? 1.0f : x); }

constexpr float kWaterIndex = 1.333f;   // refractive index of water (air: 1)

// Colormaps through 5 control points at t = 0, 1/4, ..., 1: diverging
// blue-white-red (signed values), dark-to-bright (speed), sand-green-brown
// (terrain).
__constant__ float c_maps[3][5][3] = {
    {{0.020f, 0.188f, 0.380f}, {0.263f, 0.576f, 0.765f}, {0.969f, 0.969f, 0.969f},
     {0.957f, 0.647f, 0.510f}, {0.404f, 0.000f, 0.122f}},
    {{0.050f, 0.030f, 0.200f}, {0.150f, 0.250f, 0.550f}, {0.100f, 0.600f, 0.650f},
     {0.550f, 0.850f, 0.350f}, {0.990f, 0.950f, 0.300f}},
    {{0.780f, 0.700f, 0.500f}, {0.600f, 0.650f, 0.380f}, {0.350f, 0.550f, 0.250f},
     {0.450f, 0.480f, 0.300f}, {0.550f, 0.450f, 0.350f}}};
__constant__ float c_sky_horizon[3] = {0.780f, 0.850f, 0.920f};
__constant__ float c_sky_zenith[3] = {0.250f, 0.450f, 0.800f};
__constant__ float c_water[3] = {0.020f, 0.150f, 0.200f};

__device__ __forceinline__ void colormap(int which, float t, float rgb[3])
{
    t = clamp01(t);
    const float s = ml(t, 4.0f);
    int k = __float2int_rz(s);
    if (k > 3) k = 3;
    const float f = sb(s, __int2float_rn(k));
#pragma unroll
    for (int c = 0; c < 3; c++) {
        const float a = c_maps[which][k][c], b = c_maps[which][k + 1][c];
        rgb[c] = ad(a, ml(sb(b, a), f));
    }
}

// Fresnel equations, unpolarised light from air into water.
__device__ __forceinline__ float fresnel(float cos_i)
{
    cos_i = clamp01(cos_i);
    const float sin2_i = sb(1.0f, ml(cos_i, cos_i));
    const float sin2_t = dv(sin2_i, ml(kWaterIndex, kWaterIndex));
    const float cos_t = sq(sb(1.0f, sin2_t));
    const float rs = dv(sb(cos_i, ml(kWaterIndex, cos_t)), ad(cos_i, ml(kWaterIndex, cos_t)));
    const float rp = dv(sb(ml(kWaterIndex, cos_i), cos_t), ad(ml(kWaterIndex, cos_i), cos_t));
    return ml(ad(ml(rs, rs), ml(rp, rp)), 0.5f);
}

__device__ __forceinline__ void normalize3(float v[3])
{
    const float n = sq(ad(ad(ml(v[0], v[0]), ml(v[1], v[1])), ml(v[2], v[2])));
    v[0] = dv(v[0], n);
    v[1] = dv(v[1], n);
    v[2] = dv(v[2], n);
}

__device__ __forceinline__ float dot3(const float a[3], const float b[3])
{
    return ad(ad(ml(a[0], b[0]), ml(a[1], b[1])), ml(a[2], b[2]));
}

__device__ __forceinline__ unsigned char to_byte(float c)
{
    return (unsigned char)__float2int_rz(ad(ml(clamp01(c), 255.0f), 0.5f));
}

template <typename real>
__device__ __forceinline__ float tofloat(real v) { return (float)v; }

constexpr int kRT = 32;        // pixels per tile edge
constexpr int kRS = kRT + 2;   // with a one-cell ring

template <typename real>
__global__ void __launch_bounds__(256) k_render(RenderArgs<real> A)
{
    __shared__ float sw[kRS][kRS + 1], sB[kRS][kRS + 1];   // w and Bbar with the ring (clamped)
    __shared__ float sQ[kRT][kRT + 1];                     // Q, transposed from its column-major array
    const Geo &G = A.geo;
    const int nx = G.nx, ny = G.ny;
    const int x0 = blockIdx.x * kRT, y0 = blockIdx.y * kRT;
    const int tid = threadIdx.y * 32 + threadIdx.x;
    for (int k = tid; k < kRS * kRS; k += 256) {
        const int ty = k / kRS, tx = k % kRS;
        const int i = min(max(x0 - 1 + tx, 0), nx - 1), j = min(max(y0 - 1 + ty, 0), ny - 1);
        sw[ty][tx] = tofloat(A.w[(size_t)j * G.px + i]);
        sB[ty][tx] = tofloat(bbar_at(A.Bc, G, i, j));
    }
    for (int k = tid; k < kRT * kRT; k += 256) {   // a warp reads 32 consecutive j of one column
        const int c = k / kRT, r = k % kRT;
        const int i = x0 + c, j = y0 + r;
        sQ[r][c] = (i < nx && j < ny) ? tofloat(A.Qc[(size_t)i * G.py + j]) : 0.0f;
    }
    __syncthreads();
    const float dx = A.dx, dy = A.dy, ws = A.ws;
    const cel_render_params &p = A.p;
    for (int rr = 0; rr < kRT / 8; rr++) {
        const int cx = threadIdx.x, cy = threadIdx.y + rr * 8;
        const int i = x0 + cx, j = y0 + cy;
        if (i >= nx || j >= ny) continue;
        const int sx = cx + 1, sy = cy + 1;
        const float wc = sw[sy][sx], Bc = sB[sy][sx];
        const float h = sb(wc, Bc);
        const bool wet = h > p.dry_h;
        const int iw = i > 0 ? i - 1 : i, ie = i < nx - 1 ? i + 1 : i;
        const int js = j > 0 ? j - 1 : j, jn = j < ny - 1 ? j + 1 : j;
        const float spanx = ml(__int2float_rn(ie - iw), dx), spany = ml(__int2float_rn(jn - js), dy);
        float rgb[3];
        if (!wet) {
            const float gx = spanx > 0.0f ? dv(sb(sB[sy][sx + 1], sB[sy][sx - 1]), spanx) : 0.0f;
            const float gy = spany > 0.0f ? dv(sb(sB[sy + 1][sx], sB[sy - 1][sx]), spany) : 0.0f;
            float nb[3] = {-ml(p.exaggeration, gx), -ml(p.exaggeration, gy), 1.0f};
            normalize3(nb);
            float L[3] = {p.sun[0], p.sun[1], p.sun[2]};
            normalize3(L);
            const float d = dot3(nb, L);
            const float shade = ad(0.35f, ml(0.65f, d > 0.0f ? d : 0.0f));
            colormap(2, dv(sb(Bc, p.zmin), sb(p.zmax, p.zmin)), rgb);
#pragma unroll
            for (int c = 0; c < 3; c++) rgb[c] = ml(rgb[c], shade);
        } else if (p.mode == CEL_RENDER_FRESNEL) {
            const float ec = sb(wc, ws);
            auto eta_or = [&](int ty, int tx) {
                return sb(sw[ty][tx], sB[ty][tx]) > p.dry_h ? sb(sw[ty][tx], ws) : ec;
            };
            const float eW = eta_or(sy, sx - 1), eE = eta_or(sy, sx + 1);
            const float eS = eta_or(sy - 1, sx), eN = eta_or(sy + 1, sx);
            const float gx = spanx > 0.0f ? dv(sb(eE, eW), spanx) : 0.0f;
            const float gy = spany > 0.0f ? dv(sb(eN, eS), spany) : 0.0f;
            float n[3] = {-ml(p.exaggeration, gx), -ml(p.exaggeration, gy), 1.0f};
            normalize3(n);
            float I[3] = {p.view[0], p.view[1], p.view[2]};
            normalize3(I);
            const float idn = dot3(I, n);
            const float R = fresnel(-idn);
            const float tz = clamp01(sb(I[2], ml(ml(2.0f, idn), n[2])));
            float bed[3];
            colormap(2, dv(sb(Bc, p.zmin), sb(p.zmax, p.zmin)), bed);
            const float a = dv(1.0f, ad(1.0f, ml(p.absorb, h)));
#pragma unroll
            for (int c = 0; c < 3; c++) {
                const float sky = ad(c_sky_horizon[c], ml(sb(c_sky_zenith[c], c_sky_horizon[c]), tz));
                const float refr = ad(c_water[c], ml(sb(bed[c], c_water[c]), a));
                rgb[c] = ad(ml(R, sky), ml(sb(1.0f, R), refr));
            }
        } else {
            float v;
            int map = 0;
            if (p.mode == CEL_RENDER_ETA) {
                v = sb(wc, ws);
            } else {
                const float hd = h > p.h_min ? h : p.h_min;
                const float u = dv(tofloat(A.P[(size_t)j * G.px + i]), hd), vv = dv(sQ[cy][cx], hd);
                if (p.mode == CEL_RENDER_U) {
                    v = u;
                } else if (p.mode == CEL_RENDER_V) {
                    v = vv;
                } else {
                    v = sq(ad(ml(u, u), ml(vv, vv)));
                    map = 1;
                }
            }
            colormap(map, dv(sb(v, p.vmin), sb(p.vmax, p.vmin)), rgb);
        }
        if (p.grid > 0.0f) {   // a grid line crosses the cell where floor(x / spacing) changes across it
            const bool lx = floorf(dv(ml(__int2float_rn(i + 1), dx), p.grid)) !=
                            floorf(dv(ml(__int2float_rn(i), dx), p.grid));
            const bool ly = floorf(dv(ml(__int2float_rn(j + 1), dy), p.grid)) !=
                            floorf(dv(ml(__int2float_rn(j), dy), p.grid));
            if (lx || ly) {
#pragma unroll
                for (int c = 0; c < 3; c++) rgb[c] = ml(rgb[c], 0.6f);
            }
        }
        A.rgba[(size_t)j * nx + i] = make_uchar4(to_byte(rgb[0]), to_byte(rgb[1]), to_byte(rgb[2]), 255);
    }
}

}  // namespace

template <typename real>
cudaError_t launch_render(const RenderArgs<real> &a, cudaStream_t st)
{
    dim3 grid((a.geo.nx + kRT - 1) / kRT, (a.geo.ny + kRT - 1) / kRT), block(32, 8);
    k_render<real><<<grid, block, 0, st>>>(a);
    return cudaGetLastError();
}

template cudaError_t launch_render<float>(const RenderArgs<float> &, cudaStream_t);
template cudaError_t launch_render<double>(const RenderArgs<double> &, cudaStream_t);

}  // namespace cel
