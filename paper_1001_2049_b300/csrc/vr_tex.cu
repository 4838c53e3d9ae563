// vr_tex.cu -- the texture-gather ray-march kernel (the render hot path when a
// volume has texture storage attached).
//
// Same rendering as vr_march.cu (paper §3.1 process item 3; definition in
// include/vr.h).  The difference is where the eight corners of a cell come
// from: the cube is also held as layered 2-D textures (one layer per
// frequency plane z, block-linear in x and y), and one `tld4` (four-texel
// gather) returns the 2 x 2 corners of a cell in one plane.  A sample needs
// at most two gathers (planes z0 and z0 + 1) and no address arithmetic; the
// texture unit's 2-D tiling keeps the neighbouring rays of a warp on few
// cache lines whichever way the rays run.  The gathers return the stored
// texels unfiltered, so the interpolation (x, then y, then z, FP32) is the
// kernel's own and the results are those of the definition.
//
// The gathers of the next sample are issued before the current sample is
// interpolated, which hides the texture latency behind the arithmetic.
//
// Layers: a layered texture holds at most kMaxLayers planes, so the cube is
// split into groups of planes [g*(L-1), g*(L-1) + L) that overlap by one
// plane; the plane pair (z0, z0 + 1) always lies in one group.
#include <cuda_fp16.h>

#include "vr_internal.h"

namespace vr {
namespace {

// Launch shapes the autotuner chooses from: a block of BX x BY rays (one
// thread each), warps holding PX x PY packets of neighbouring rays, and the
// minimum number of resident blocks per SM the register budget must allow.
struct Shape {
    int bx, by, px, py, minb;
};
constexpr Shape kShapes[] = {
    {16, 16, 8, 4, 1}, {16, 16, 8, 4, 6}, {32, 8, 8, 4, 5}, {16, 16, 16, 2, 5},
    {16, 16, 4, 8, 5}, {8, 8, 8, 4, 16},
};
constexpr int kNumShapes = sizeof(kShapes) / sizeof(kShapes[0]);

__device__ __forceinline__ float lerpf(float a, float b, float f) { return fmaf(f, b - a, a); }

// Four texels around (x, y) of a layer: with x = i + 1, y = j + 1 (texel
// centres at +0.5) the footprint is texels i..i+1, j..j+1, returned as
// (i, j+1), (i+1, j+1), (i+1, j), (i, j).
template <int DT>
__device__ __forceinline__ float4 gather(cudaTextureObject_t t, int layer, float x, float y);

template <>
__device__ __forceinline__ float4 gather<VR_F32>(cudaTextureObject_t t, int layer, float x,
                                                 float y)
{
    float4 r;
    asm volatile("tld4.r.a2d.v4.f32.f32 {%0, %1, %2, %3}, [%4, {%5, %6, %7, %7}];"
                 : "=f"(r.x), "=f"(r.y), "=f"(r.z), "=f"(r.w)
                 : "l"(t), "r"(layer), "f"(x), "f"(y));
    return r;
}

template <>
__device__ __forceinline__ float4 gather<VR_F16>(cudaTextureObject_t t, int layer, float x,
                                                 float y)
{
    return gather<VR_F32>(t, layer, x, y);   // half texels are returned as floats
}

template <>
__device__ __forceinline__ float4 gather<VR_I8>(cudaTextureObject_t t, int layer, float x,
                                                float y)
{
    int q0, q1, q2, q3;
    asm volatile("tld4.r.a2d.v4.s32.f32 {%0, %1, %2, %3}, [%4, {%5, %6, %7, %7}];"
                 : "=r"(q0), "=r"(q1), "=r"(q2), "=r"(q3)
                 : "l"(t), "r"(layer), "f"(x), "f"(y));
    return make_float4((float)q0, (float)q1, (float)q2, (float)q3);
}

struct Ray {
    float ox, oy, oz, dx, dy, dz, te;
    int K;
};

__device__ __forceinline__ Ray setup_ray(const MarchParams& P, const vr_camera& c, int px, int py,
                                         int k_max)
{
    Ray r;
    const float u = ((float)px + 0.5f) - 0.5f * (float)P.w;
    const float v = ((float)py + 0.5f) - 0.5f * (float)P.h;
    float d0, d1, d2;
    if (c.proj == VR_ORTHO) {
        r.ox = fmaf(v, c.dv[0], fmaf(u, c.du[0], c.eye[0]));
        r.oy = fmaf(v, c.dv[1], fmaf(u, c.du[1], c.eye[1]));
        r.oz = fmaf(v, c.dv[2], fmaf(u, c.du[2], c.eye[2]));
        d0 = c.fwd[0];
        d1 = c.fwd[1];
        d2 = c.fwd[2];
    } else {
        r.ox = c.eye[0];
        r.oy = c.eye[1];
        r.oz = c.eye[2];
        d0 = fmaf(v, c.dv[0], fmaf(u, c.du[0], c.fwd[0]));
        d1 = fmaf(v, c.dv[1], fmaf(u, c.du[1], c.fwd[1]));
        d2 = fmaf(v, c.dv[2], fmaf(u, c.du[2], c.fwd[2]));
    }
    const float nrm = sqrtf(fmaf(d0, d0, fmaf(d1, d1, d2 * d2)));
    r.dx = d0 / nrm;
    r.dy = d1 / nrm;
    r.dz = d2 / nrm;
    r.K = 0;
    r.te = 0.0f;
    if (!(nrm > 0.0f) || !isfinite(nrm)) return r;
    float tn = -INFINITY, tf = INFINITY;
    bool inside = true;
    const float o[3] = {r.ox, r.oy, r.oz};
    const float d[3] = {r.dx, r.dy, r.dz};
    const float hi[3] = {P.hix, P.hiy, P.hiz};
#pragma unroll
    for (int a = 0; a < 3; ++a) {
        if (d[a] != 0.0f) {
            const float ta = (0.0f - o[a]) / d[a];
            const float tb = (hi[a] - o[a]) / d[a];
            tn = fmaxf(tn, fminf(ta, tb));
            tf = fminf(tf, fmaxf(ta, tb));
        } else if (o[a] < 0.0f || o[a] > hi[a]) {
            inside = false;
        }
    }
    const float te = fmaxf(tn, 0.0f);
    if (inside && tf >= te) {
        const float q = floorf((tf - te) / P.step);
        r.K = (q < (float)k_max) ? (int)q + 1 : k_max;
        r.te = te;
    }
    return r;
}

// Decode int8 codes of plane z (scale/offset); identity for float storage.
template <int DT>
__device__ __forceinline__ float4 decode(const TexParams& T, float4 q, int z)
{
    if (DT != VR_I8) return q;
    const float s = __ldg(T.scale + z), o = __ldg(T.offset + z);
    return make_float4(fmaf(q.x, s, o), fmaf(q.y, s, o), fmaf(q.z, s, o), fmaf(q.w, s, o));
}

// The two planes z and z + 1 of the cell whose x/y corner is texel (x-1, y-1).
template <int DT, bool MULTI>
__device__ __forceinline__ void cell(const TexParams& T, cudaTextureObject_t t0, int z, float x,
                                     float y, float4& q0, float4& q1)
{
    if (!MULTI) {
        q0 = gather<DT>(t0, z, x, y);
        q1 = gather<DT>(t0, z + 1, x, y);
    } else {
        // plane pair (z, z + 1) lies in group min(z / (L-1), last)
        const int g = min(z / (kMaxLayers - 1), T.n_groups - 1);
        const cudaTextureObject_t t = T.tex[g];
        const int l = z - g * (kMaxLayers - 1);
        q0 = gather<DT>(t, l, x, y);
        q1 = gather<DT>(t, l + 1, x, y);
    }
    q0 = decode<DT>(T, q0, z);
    q1 = decode<DT>(T, q1, z + 1);
}

// Corners of the cell of sample geometry `n` given the cell `c` whose corners
// (c0, c1) are held: nothing is fetched when the cell is the same, one plane
// when only z moved by one, both planes otherwise.  The texture return path
// is what bounds this kernel, so every gather saved counts.
template <int DT, bool MULTI, typename G>
__device__ __forceinline__ void next_cell(const TexParams& T, cudaTextureObject_t t0, const G& c,
                                          const float4& c0, const float4& c1, const G& n,
                                          float4& n0, float4& n1)
{
    if (n.gx == c.gx && n.gy == c.gy) {
        if (n.iz == c.iz) {
            n0 = c0;
            n1 = c1;
            return;
        }
        if (n.iz == c.iz + 1) {
            float4 u0, u1;
            n0 = c1;
            if (!MULTI) {
                n1 = decode<DT>(T, gather<DT>(t0, n.iz + 1, n.gx, n.gy), n.iz + 1);
            } else {
                cell<DT, MULTI>(T, t0, n.iz, n.gx, n.gy, u0, u1);
                n1 = u1;
            }
            return;
        }
    }
    cell<DT, MULTI>(T, t0, n.iz, n.gx, n.gy, n0, n1);
}

// Per-sample geometry: the gather coordinates of the cell and the weights.
// x and y are not clamped to the box: a position just outside a face (by
// rounding) has both its corners clamped to the edge texel by the texture
// unit, which gives the edge value exactly as clamping the position would.
// z is the layer index and is clamped explicitly (cell in [0, nz - 2],
// weight in [0, 1]).
struct Geo {
    float gx, gy;     // gather coordinates (cell corner + 1)
    float fx, fy, fz;
    int iz;
};

__device__ __forceinline__ Geo geo(const MarchParams& P, const Ray& r, float kf)
{
    Geo g;
    const float t = fmaf(kf, P.step, r.te);
    const float px = fmaf(t, r.dx, r.ox), py = fmaf(t, r.dy, r.oy), pz = fmaf(t, r.dz, r.oz);
    const float flx = floorf(px), fly = floorf(py);
    const float flz = fminf(fmaxf(floorf(pz), 0.0f), P.hiz - 1.0f);
    g.gx = flx + 1.0f;
    g.gy = fly + 1.0f;
    g.fx = px - flx;
    g.fy = py - fly;
    g.fz = fminf(fmaxf(pz - flz, 0.0f), 1.0f);
    g.iz = (int)flz;
    return g;
}

__device__ __forceinline__ float interp(const float4& q0, const float4& q1, const Geo& g)
{
    // q = ((x0,y1), (x1,y1), (x1,y0), (x0,y0)) of planes z0 (q0) and z0 + 1 (q1)
    const float y0z0 = lerpf(q0.w, q0.z, g.fx);
    const float y1z0 = lerpf(q0.x, q0.y, g.fx);
    const float y0z1 = lerpf(q1.w, q1.z, g.fx);
    const float y1z1 = lerpf(q1.x, q1.y, g.fx);
    return lerpf(lerpf(y0z0, y1z0, g.fy), lerpf(y0z1, y1z1, g.fy), g.fz);
}

// Accumulate one sample; returns true when the ray terminates.
template <int MODE>
struct Acc {
    float r = 0.0f, g = 0.0f, b = 0.0f, A = 0.0f;
    float m = (MODE == VR_MIP) ? -INFINITY : 0.0f;

    __device__ __forceinline__ bool add(const MarchParams& P, const float4* __restrict__ lut,
                                        float s)
    {
        if (MODE == VR_MIP) {
            m = fmaxf(m, s);
            return false;
        }
        if (MODE == VR_SUM) {
            m = fmaf(s, P.step, m);
            return false;
        }
        if (!(s >= P.clip)) return false;
        const float x = fminf(fmaxf((s - P.v_lo) * P.lut_scale, 0.0f), P.lut_max);
        const int i = min((int)x, P.n_lut - 2);
        const float f = x - (float)i;
        const float4 a = lut[i], c = lut[i + 1];
        const float alpha = lerpf(a.w, c.w, f);
        const float wgt = (1.0f - A) * alpha;
        r = fmaf(wgt, lerpf(a.x, c.x, f), r);
        g = fmaf(wgt, lerpf(a.y, c.y, f), g);
        b = fmaf(wgt, lerpf(a.z, c.z, f), b);
        A += wgt;
        return A >= P.term_alpha;
    }
};

// The gathers of sample k + 1 are issued before sample k is interpolated, so
// the texture latency overlaps the arithmetic of the current sample.  The
// loop is unrolled twice with two register sets that swap roles, so a
// pending gather result is only copied when the next sample reuses it.
template <int DT, int MODE, bool MULTI, int CFG>
__global__ void __launch_bounds__(kShapes[CFG].bx * kShapes[CFG].by, kShapes[CFG].minb)
    tex_kernel(const __grid_constant__ MarchParams P, const __grid_constant__ TexParams T)
{
    constexpr Shape S = kShapes[CFG];
    __shared__ float4 s_lut[VR_MAX_LUT];
    if (MODE == VR_COMPOSITE) {
        for (int i = threadIdx.x; i < P.n_lut; i += blockDim.x) s_lut[i] = P.lut[i];
        __syncthreads();
    }
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    constexpr int wpr = S.bx / S.px;                 // warps per block row
    const int px = blockIdx.x * S.bx + (warp % wpr) * S.px + (lane % S.px);
    const int py = blockIdx.y * S.by + (warp / wpr) * S.py + (lane / S.px);
    const int view = blockIdx.z;
    const bool valid = px < P.w && py < P.h;
    const cudaTextureObject_t t0 = T.tex[0];
    unsigned count = 0;
    if (valid) {
        const Ray r = setup_ray(P, P.cams[view], px, py, T.k_max);
        const size_t pix = ((size_t)view * P.h + py) * P.w + px;
        Acc<MODE> acc;
        int k = 0;
        if (r.K > 0) {
            Geo ga = geo(P, r, 0.0f), gb;
            float4 a0, a1, b0, b1;
            cell<DT, MULTI>(T, t0, ga.iz, ga.gx, ga.gy, a0, a1);
            float kf = 1.0f;
            for (;;) {
                gb = geo(P, r, kf);
                next_cell<DT, MULTI>(T, t0, ga, a0, a1, gb, b0, b1);
                ++k;
                if (acc.add(P, s_lut, interp(a0, a1, ga)) || k >= r.K) break;
                kf += 1.0f;
                ga = geo(P, r, kf);
                next_cell<DT, MULTI>(T, t0, gb, b0, b1, ga, a0, a1);
                ++k;
                if (acc.add(P, s_lut, interp(b0, b1, gb)) || k >= r.K) break;
                kf += 1.0f;
            }
        }
        count = (unsigned)k;
        if (MODE == VR_COMPOSITE)
            reinterpret_cast<float4*>(P.out)[pix] = make_float4(acc.r, acc.g, acc.b, acc.A);
        else
            P.out[pix] = acc.m;
    }
    if (P.samples) {
        const unsigned tot = __reduce_add_sync(0xffffffffu, count);
        if (lane == 0 && tot) atomicAdd(P.samples, (unsigned long long)tot);
    }
}

template <int DT, int MODE, bool MULTI, int CFG>
cudaError_t launch_c(const MarchParams& p, const TexParams& t, cudaStream_t s)
{
    constexpr Shape S = kShapes[CFG];
    dim3 grid((unsigned)((p.w + S.bx - 1) / S.bx), (unsigned)((p.h + S.by - 1) / S.by),
              (unsigned)p.n_views);
    tex_kernel<DT, MODE, MULTI, CFG><<<grid, S.bx * S.by, 0, s>>>(p, t);
    return cudaGetLastError();
}

template <int DT, int MODE, bool MULTI>
cudaError_t launch_m(const MarchParams& p, const TexParams& t, int cfg, cudaStream_t s)
{
    switch (cfg) {
    case 1: return launch_c<DT, MODE, MULTI, 1>(p, t, s);
    case 2: return launch_c<DT, MODE, MULTI, 2>(p, t, s);
    case 3: return launch_c<DT, MODE, MULTI, 3>(p, t, s);
    case 4: return launch_c<DT, MODE, MULTI, 4>(p, t, s);
    case 5: return launch_c<DT, MODE, MULTI, 5>(p, t, s);
    default: return launch_c<DT, MODE, MULTI, 0>(p, t, s);
    }
}
static_assert(kNumShapes == 6, "launch_m lists every shape");

template <int DT, int MODE>
cudaError_t launch_t(const MarchParams& p, const TexParams& t, int cfg, cudaStream_t s)
{
    return t.n_groups > 1 ? launch_m<DT, MODE, true>(p, t, cfg, s)
                          : launch_m<DT, MODE, false>(p, t, cfg, s);
}

template <int DT>
cudaError_t launch_dt(const MarchParams& p, const TexParams& t, int mode, int cfg,
                      cudaStream_t s)
{
    switch (mode) {
    case VR_MIP: return launch_t<DT, VR_MIP>(p, t, cfg, s);
    case VR_COMPOSITE: return launch_t<DT, VR_COMPOSITE>(p, t, cfg, s);
    default: return launch_t<DT, VR_SUM>(p, t, cfg, s);
    }
}

// Copy planes [z0, z1) from the bricks into texture group g (surface writes).
template <typename T>
__global__ void __launch_bounds__(256) fill_kernel(const T* __restrict__ bricks, VolumeGeom g,
                                                   cudaSurfaceObject_t surf, int layer0, int z0,
                                                   int z1)
{
    const int x = blockIdx.x * 32 + (threadIdx.x & 31);
    const int y = blockIdx.y * 8 + (threadIdx.x >> 5);
    if (x >= g.nx || y >= g.ny) return;
    for (int z = z0 + blockIdx.z; z < z1; z += gridDim.z) {
        const size_t brick = ((size_t)(z >> kBrickShift) * g.nby + (y >> kBrickShift)) * g.nbx +
                             (x >> kBrickShift);
        const T v = bricks[brick * kBrickVoxels + ((z & 31) << 10) + ((y & 31) << 5) + (x & 31)];
        surf2DLayeredwrite(v, surf, x * (int)sizeof(T), y, z - layer0);
    }
}

}  // namespace

cudaError_t launch_tex(const MarchParams& p, const TexParams& t, int dtype, int mode, int cfg,
                       cudaStream_t s)
{
    if (cfg < 0 || cfg >= kNumShapes) cfg = 0;
    switch (dtype) {
    case VR_F32: return launch_dt<VR_F32>(p, t, mode, cfg, s);
    case VR_F16: return launch_dt<VR_F16>(p, t, mode, cfg, s);
    default: return launch_dt<VR_I8>(p, t, mode, cfg, s);
    }
}

int tex_shape_count() { return kNumShapes; }

void tex_shape(int cfg, int* bx, int* by, int* px, int* py, int* minb)
{
    const Shape& sh = kShapes[cfg];
    *bx = sh.bx;
    *by = sh.by;
    *px = sh.px;
    *py = sh.py;
    *minb = sh.minb;
}

cudaError_t fill_texture_group(const Volume& v, cudaSurfaceObject_t surf, int layer0, int z0,
                               int z1, cudaStream_t s)
{
    dim3 grid((unsigned)((v.g.nx + 31) / 32), (unsigned)((v.g.ny + 7) / 8),
              (unsigned)((z1 - z0) < 1024 ? (z1 - z0) : 1024));
    switch (v.dtype) {
    case VR_F32:
        fill_kernel<float><<<grid, 256, 0, s>>>((const float*)v.bricks, v.g, surf, layer0, z0, z1);
        break;
    case VR_F16:   // binary16 bit patterns moved as 16-bit words
        fill_kernel<unsigned short><<<grid, 256, 0, s>>>((const unsigned short*)v.bricks, v.g,
                                                         surf, layer0, z0, z1);
        break;
    default:
        fill_kernel<signed char><<<grid, 256, 0, s>>>((const signed char*)v.bricks, v.g, surf,
                                                      layer0, z0, z1);
        break;
    }
    return cudaGetLastError();
}

}  // namespace vr
