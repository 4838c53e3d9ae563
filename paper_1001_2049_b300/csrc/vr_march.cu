// vr_march.cu -- the ray-marching kernels (the render hot path).
//
// Paper §3.1 process item 3: each GPU maps every output pixel to RGBA through
// a pre-selected transfer function by casting a ray through the cube.  One
// thread marches one ray; a warp holds an 8 x 4 packet of neighbouring
// pixels, so its rays stay close together in the cube and finish at similar
// depths (a warp leaves the sample loop when all 32 rays are done).
//
// Per ray (all single precision, see include/vr.h for the definition):
//   camera -> ray, slab entry/exit, K = floor((t_exit - t_entry)/step) + 1,
//   for k < K: t_k = fma(k, step, t_entry) from the integer k, p = clamp(
//   fma(t_k, d, o)), eight corners from the bricked cube, trilinear (x, y,
//   z), then MIP max / SUM / clip + table lookup + front-to-back compositing
//   with early termination.
//
// Memory: the cube stays in HBM in 32^3 bricks; corners are gathered with
// read-only loads.  A cell whose corners straddle a brick boundary uses the
// per-axis strides of the neighbouring brick.  The (opacity-corrected)
// transfer table is copied from the kernel parameters into shared memory.
#include <cstdlib>

#include <cuda_fp16.h>

#include "vr_internal.h"

namespace vr {
namespace {

constexpr int kBlockX = 16, kBlockY = 16;     // 256 threads, 8 warps of 8x4 rays

template <int DT>
struct Voxel;

template <>
struct Voxel<VR_F32> {
    __device__ static float load(const void* b, size_t i) {
        return __ldg(static_cast<const float*>(b) + i);
    }
};

template <>
struct Voxel<VR_F16> {
    __device__ static float load(const void* b, size_t i) {
        return __half2float(__ldg(static_cast<const __half*>(b) + i));
    }
};

template <>
struct Voxel<VR_I8> {
    __device__ static float load(const void* b, size_t i) {
        return (float)__ldg(static_cast<const signed char*>(b) + i);
    }
};

__device__ __forceinline__ float lerpf(float a, float b, float f) { return fmaf(f, b - a, a); }

// Trilinear sample at a point already clamped to the box.
template <int DT>
__device__ __forceinline__ float sample(const MarchParams& P, float px, float py, float pz)
{
    const VolumeGeom& g = P.g;
    const int ix = min((int)px, g.nx - 2);
    const int iy = min((int)py, g.ny - 2);
    const int iz = min((int)pz, g.nz - 2);
    const float fx = px - (float)ix;
    const float fy = py - (float)iy;
    const float fz = pz - (float)iz;
    const size_t brick = ((size_t)(iz >> kBrickShift) * g.nby + (iy >> kBrickShift)) * g.nbx +
                         (ix >> kBrickShift);
    const size_t base = brick * kBrickVoxels + ((iz & 31) << 10) + ((iy & 31) << 5) + (ix & 31);
    const size_t sx = ((ix & 31) == 31) ? (size_t)(kBrickVoxels - 31) : 1;
    const size_t sy = ((iy & 31) == 31) ? (size_t)g.nbx * kBrickVoxels - 31 * 32 : 32;
    const size_t sz = ((iz & 31) == 31) ? (size_t)g.nbx * g.nby * kBrickVoxels - 31 * 1024 : 1024;
    float c000 = Voxel<DT>::load(P.bricks, base);
    float c100 = Voxel<DT>::load(P.bricks, base + sx);
    float c010 = Voxel<DT>::load(P.bricks, base + sy);
    float c110 = Voxel<DT>::load(P.bricks, base + sx + sy);
    float c001 = Voxel<DT>::load(P.bricks, base + sz);
    float c101 = Voxel<DT>::load(P.bricks, base + sz + sx);
    float c011 = Voxel<DT>::load(P.bricks, base + sz + sy);
    float c111 = Voxel<DT>::load(P.bricks, base + sz + sx + sy);
    if (DT == VR_I8) {
        // decode each corner with its own plane's scale and offset first
        const float s0 = __ldg(P.scale + iz), o0 = __ldg(P.offset + iz);
        const float s1 = __ldg(P.scale + iz + 1), o1 = __ldg(P.offset + iz + 1);
        c000 = fmaf(c000, s0, o0); c100 = fmaf(c100, s0, o0);
        c010 = fmaf(c010, s0, o0); c110 = fmaf(c110, s0, o0);
        c001 = fmaf(c001, s1, o1); c101 = fmaf(c101, s1, o1);
        c011 = fmaf(c011, s1, o1); c111 = fmaf(c111, s1, o1);
    }
    const float y0z0 = lerpf(c000, c100, fx);
    const float y1z0 = lerpf(c010, c110, fx);
    const float y0z1 = lerpf(c001, c101, fx);
    const float y1z1 = lerpf(c011, c111, fx);
    const float z0 = lerpf(y0z0, y1z0, fy);
    const float z1 = lerpf(y0z1, y1z1, fy);
    return lerpf(z0, z1, fz);
}

struct Ray {
    float ox, oy, oz, dx, dy, dz;
    float t_entry;
    int K;
};

// Camera -> ray -> box -> sample count.  A degenerate direction gives K = 0.
__device__ __forceinline__ Ray setup_ray(const MarchParams& P, const vr_camera& c, int px,
                                         int py, int k_max)
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
    r.t_entry = 0.0f;
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
            inside = false;          // parallel to this axis and outside it
        }
    }
    const float te = fmaxf(tn, 0.0f);
    if (inside && tf >= te) {
        const float q = floorf((tf - te) / P.step);
        r.K = (q < (float)k_max) ? (int)q + 1 : k_max;
        r.t_entry = te;
    }
    return r;
}

template <int DT, int MODE, bool COUNT>
__global__ void __launch_bounds__(kBlockX * kBlockY) march_kernel(const __grid_constant__ MarchParams P,
                                                                  int k_max)
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
        const Ray r = setup_ray(P, P.cams[view], px, py, k_max);
        const size_t pix = ((size_t)view * P.h + py) * P.w + px;
        if (MODE == VR_COMPOSITE) {
            float cr = 0.0f, cg = 0.0f, cb = 0.0f, A = 0.0f;
            int k = 0;
            for (; k < r.K; ++k) {
                const float t = fmaf((float)k, P.step, r.t_entry);
                const float qx = fminf(fmaxf(fmaf(t, r.dx, r.ox), 0.0f), P.hix);
                const float qy = fminf(fmaxf(fmaf(t, r.dy, r.oy), 0.0f), P.hiy);
                const float qz = fminf(fmaxf(fmaf(t, r.dz, r.oz), 0.0f), P.hiz);
                const float s = sample<DT>(P, qx, qy, qz);
                if (s >= P.clip) {
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
            reinterpret_cast<float4*>(P.out)[pix] = make_float4(cr, cg, cb, A);
        } else {
            float m = (MODE == VR_MIP) ? -INFINITY : 0.0f;
            for (int k = 0; k < r.K; ++k) {
                const float t = fmaf((float)k, P.step, r.t_entry);
                const float qx = fminf(fmaxf(fmaf(t, r.dx, r.ox), 0.0f), P.hix);
                const float qy = fminf(fmaxf(fmaf(t, r.dy, r.oy), 0.0f), P.hiy);
                const float qz = fminf(fmaxf(fmaf(t, r.dz, r.oz), 0.0f), P.hiz);
                const float s = sample<DT>(P, qx, qy, qz);
                if (MODE == VR_MIP)
                    m = fmaxf(m, s);
                else
                    m = fmaf(s, P.step, m);
            }
            count = (unsigned)r.K;
            P.out[pix] = m;
        }
    }
    if (COUNT) {
        const unsigned tot = __reduce_add_sync(0xffffffffu, count);
        if (lane == 0 && tot) atomicAdd(P.samples, (unsigned long long)tot);
    }
}

template <int DT, int MODE>
cudaError_t launch_t(const MarchParams& p, cudaStream_t s, int k_max)
{
    dim3 grid((unsigned)((p.w + kBlockX - 1) / kBlockX), (unsigned)((p.h + kBlockY - 1) / kBlockY),
              (unsigned)p.n_views);
    if (p.samples)
        march_kernel<DT, MODE, true><<<grid, kBlockX * kBlockY, 0, s>>>(p, k_max);
    else
        march_kernel<DT, MODE, false><<<grid, kBlockX * kBlockY, 0, s>>>(p, k_max);
    return cudaGetLastError();
}

template <int DT>
cudaError_t launch_dt(const MarchParams& p, int mode, cudaStream_t s, int k_max)
{
    switch (mode) {
    case VR_MIP: return launch_t<DT, VR_MIP>(p, s, k_max);
    case VR_COMPOSITE: return launch_t<DT, VR_COMPOSITE>(p, s, k_max);
    default: return launch_t<DT, VR_SUM>(p, s, k_max);
    }
}

}  // namespace

// Slab window plan (measured on the 1024^3 orbit views): 4 cells per slab,
// a one-voxel margin, slabs along y or z when that direction component is at
// least 0.25, the window grown 10 % over the reach of a tile, at most 50 KB.
constexpr int kSlabCells = 4;
constexpr int kSlabMargin = 1;
constexpr float kSlabMinAxis = 0.25f;
constexpr double kSlabGrow = 1.10;
constexpr int kSlabWindowKB = 50;

bool plan_slab(const MarchParams& p, SlabConfig* c)
{
    // largest spacing between neighbouring rays inside the cube: the pixel
    // step at the farthest cube corner (perspective) or the pixel step itself
    double sp = 0.0;
    for (int v = 0; v < p.n_views; ++v) {
        const vr_camera& cam = p.cams[v];
        const double du = sqrt((double)cam.du[0] * cam.du[0] + (double)cam.du[1] * cam.du[1] +
                               (double)cam.du[2] * cam.du[2]);
        const double dv = sqrt((double)cam.dv[0] * cam.dv[0] + (double)cam.dv[1] * cam.dv[1] +
                               (double)cam.dv[2] * cam.dv[2]);
        double s = du > dv ? du : dv;
        if (cam.proj == VR_PERSP) {
            const double f = sqrt((double)cam.fwd[0] * cam.fwd[0] + (double)cam.fwd[1] * cam.fwd[1] +
                                  (double)cam.fwd[2] * cam.fwd[2]);
            double tmax = 0.0;
            for (int i = 0; i < 8; ++i) {
                const double cx = (i & 1) ? p.hix : 0.0, cy = (i & 2) ? p.hiy : 0.0,
                             cz = (i & 4) ? p.hiz : 0.0;
                const double dx = cx - cam.eye[0], dy = cy - cam.eye[1], dz = cz - cam.eye[2];
                const double t = sqrt(dx * dx + dy * dy + dz * dz);
                if (t > tmax) tmax = t;
            }
            s = s * tmax / f;
        }
        if (s > sp) sp = s;
    }
    c->S = kSlabCells;
    c->margin = kSlabMargin;
    c->min_axis = kSlabMinAxis;
    c->ea_pitch = (c->S + 1) | 1;
    // one window buffer: the bigger of the plane footprint a 16 x 16 tile can
    // reach (ray spacing, slant across the slab, margins) and a floor, within
    // a budget that keeps two blocks per SM
    const double grow = kSlabGrow;
    const double side = 16.0 * sp * grow + 3.0 * (c->S + 1) + 2.0 * c->margin + 8.0;
    const double want = side * side * (c->S + 1);
    const int budget = kSlabWindowKB * 1024 / 4;
    int elems = (int)(want < budget ? want : budget);
    if (elems < 4096) elems = 4096;
    c->win_elems = (elems + 3) & ~3;
    c->eb_max = 0;
    c->ec_max = 0;
    const double diag = sqrt((double)p.hix * p.hix + (double)p.hiy * p.hiy + (double)p.hiz * p.hiz);
    c->k_max = (int)(diag / p.step) + 2;
    c->smem_bytes = slab_smem_bytes(*c);
    return c->S >= 1 && c->S <= 7 && c->smem_bytes <= 220 * 1024;
}

cudaError_t launch_march(const MarchParams& p, int dtype, int mode, cudaStream_t s)
{
    // a ray crosses at most the box diagonal: bound the loop count from it
    const double diag = sqrt((double)p.hix * p.hix + (double)p.hiy * p.hiy + (double)p.hiz * p.hiz);
    const int k_max = (int)(diag / p.step) + 2;
    if (dtype == VR_F32) {
        SlabConfig c;
        if (plan_slab(p, &c)) return launch_slab(p, c, mode, s);
    }
    switch (dtype) {
    case VR_F32: return launch_dt<VR_F32>(p, mode, s, k_max);
    case VR_F16: return launch_dt<VR_F16>(p, mode, s, k_max);
    default: return launch_dt<VR_I8>(p, mode, s, k_max);
    }
}

}  // namespace vr
