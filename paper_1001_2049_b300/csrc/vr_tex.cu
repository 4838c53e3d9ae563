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
// A ray keeps its last cell's corners in registers: a sample in the same cell
// fetches nothing, and a step to the next plane along z with the same x/y cell
// fetches one plane instead of two.
//
// Layers: a layered texture holds at most kMaxLayers planes, so the cube is
// split into groups of planes [g*(L-1), g*(L-1) + L) that overlap by one
// plane; the plane pair (z0, z0 + 1) always lies in one group.
#include <cuda_fp16.h>

#include "vr_internal.h"

namespace vr {
namespace {

constexpr int kBlockX = 16, kBlockY = 16;

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

template <int DT>
__device__ __forceinline__ float4 plane(const TexParams& T, int z, float x, float y)
{
    const int g = min(z / (kMaxLayers - 1), T.n_groups - 1);
    const float4 q = gather<DT>(T.tex[g], z - g * (kMaxLayers - 1), x, y);
    return decode<DT>(T, q, z);
}

template <int DT, int MODE, bool COUNT>
__global__ void __launch_bounds__(kBlockX * kBlockY) tex_kernel(const __grid_constant__ MarchParams P,
                                                                const __grid_constant__ TexParams T)
{
    __shared__ float4 s_lut[VR_MAX_LUT];
    if (MODE == VR_COMPOSITE) {
        for (int i = threadIdx.x; i < P.n_lut; i += blockDim.x) s_lut[i] = P.lut[i];
        __syncthreads();
    }
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int px = blockIdx.x * kBlockX + (warp & 1) * 8 + (lane & 7);
    const int py = blockIdx.y * kBlockY + (warp >> 1) * 4 + (lane >> 3);
    const int view = blockIdx.z;
    const bool valid = px < P.w && py < P.h;
    unsigned count = 0;
    if (valid) {
        const Ray r = setup_ray(P, P.cams[view], px, py, T.k_max);
        const size_t pix = ((size_t)view * P.h + py) * P.w + px;
        float cr = 0.0f, cg = 0.0f, cb = 0.0f, A = 0.0f;
        float m = (MODE == VR_MIP) ? -INFINITY : 0.0f;
        // cached cell: (cx, cy) in x/y, cz in z; q0/q1 its planes cz, cz + 1
        float cx = -2.0f, cy = -2.0f;
        int cz = -2;
        float4 q0 = make_float4(0, 0, 0, 0), q1 = q0;
        float kf = 0.0f;
        int k = 0;
        for (; k < r.K; ++k, kf += 1.0f) {
            const float t = fmaf(kf, P.step, r.te);
            const float ppx = fminf(fmaxf(fmaf(t, r.dx, r.ox), 0.0f), P.hix);
            const float ppy = fminf(fmaxf(fmaf(t, r.dy, r.oy), 0.0f), P.hiy);
            const float ppz = fminf(fmaxf(fmaf(t, r.dz, r.oz), 0.0f), P.hiz);
            const float flx = floorf(ppx), fly = floorf(ppy), flz = floorf(ppz);
            // z cell with the last pair of planes kept inside the cube
            const int iz = min((int)flz, P.g.nz - 2);
            if (flx != cx || fly != cy) {
                q0 = plane<DT>(T, iz, flx + 1.0f, fly + 1.0f);
                q1 = plane<DT>(T, iz + 1, flx + 1.0f, fly + 1.0f);
                cx = flx;
                cy = fly;
                cz = iz;
            } else if (iz != cz) {
                if (iz == cz + 1) {
                    q0 = q1;
                    q1 = plane<DT>(T, iz + 1, flx + 1.0f, fly + 1.0f);
                } else if (iz == cz - 1) {
                    q1 = q0;
                    q0 = plane<DT>(T, iz, flx + 1.0f, fly + 1.0f);
                } else {
                    q0 = plane<DT>(T, iz, flx + 1.0f, fly + 1.0f);
                    q1 = plane<DT>(T, iz + 1, flx + 1.0f, fly + 1.0f);
                }
                cz = iz;
            }
            // texels beyond the last column/row are clamped copies with weight 0
            const float fx = ppx - flx, fy = ppy - fly, fz = ppz - (float)iz;
            const float y0z0 = lerpf(q0.w, q0.z, fx);
            const float y1z0 = lerpf(q0.x, q0.y, fx);
            const float y0z1 = lerpf(q1.w, q1.z, fx);
            const float y1z1 = lerpf(q1.x, q1.y, fx);
            const float s = lerpf(lerpf(y0z0, y1z0, fy), lerpf(y0z1, y1z1, fy), fz);
            if (MODE == VR_MIP) {
                m = fmaxf(m, s);
            } else if (MODE == VR_SUM) {
                m = fmaf(s, P.step, m);
            } else if (s >= P.clip) {
                const float x = fminf(fmaxf((s - P.v_lo) * P.lut_scale, 0.0f), P.lut_max);
                const int i = min((int)x, P.n_lut - 2);
                const float f = x - (float)i;
                const float4 a = s_lut[i], b = s_lut[i + 1];
                const float alpha = lerpf(a.w, b.w, f);
                const float wgt = (1.0f - A) * alpha;
                cr = fmaf(wgt, lerpf(a.x, b.x, f), cr);
                cg = fmaf(wgt, lerpf(a.y, b.y, f), cg);
                cb = fmaf(wgt, lerpf(a.z, b.z, f), cb);
                A += wgt;
                if (A >= P.term_alpha) {
                    ++k;
                    break;
                }
            }
        }
        count = (unsigned)k;
        if (MODE == VR_COMPOSITE)
            reinterpret_cast<float4*>(P.out)[pix] = make_float4(cr, cg, cb, A);
        else
            P.out[pix] = m;
    }
    if (COUNT) {
        const unsigned tot = __reduce_add_sync(0xffffffffu, count);
        if (lane == 0 && tot) atomicAdd(P.samples, (unsigned long long)tot);
    }
}

template <int DT, int MODE>
cudaError_t launch_t(const MarchParams& p, const TexParams& t, cudaStream_t s)
{
    dim3 grid((unsigned)((p.w + kBlockX - 1) / kBlockX), (unsigned)((p.h + kBlockY - 1) / kBlockY),
              (unsigned)p.n_views);
    if (p.samples)
        tex_kernel<DT, MODE, true><<<grid, kBlockX * kBlockY, 0, s>>>(p, t);
    else
        tex_kernel<DT, MODE, false><<<grid, kBlockX * kBlockY, 0, s>>>(p, t);
    return cudaGetLastError();
}

template <int DT>
cudaError_t launch_dt(const MarchParams& p, const TexParams& t, int mode, cudaStream_t s)
{
    switch (mode) {
    case VR_MIP: return launch_t<DT, VR_MIP>(p, t, s);
    case VR_COMPOSITE: return launch_t<DT, VR_COMPOSITE>(p, t, s);
    default: return launch_t<DT, VR_SUM>(p, t, s);
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

cudaError_t launch_tex(const MarchParams& p, const TexParams& t, int dtype, int mode,
                       cudaStream_t s)
{
    switch (dtype) {
    case VR_F32: return launch_dt<VR_F32>(p, t, mode, s);
    case VR_F16: return launch_dt<VR_F16>(p, t, mode, s);
    default: return launch_dt<VR_I8>(p, t, mode, s);
    }
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
