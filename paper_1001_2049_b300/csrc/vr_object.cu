// vr_object.cu -- object-order MIP: sub-cubes staged in shared memory once
// and rendered for every view of a launch.
//
// The paper partitions the cube into sub-cubes and ray casts each sub-cube
// into an image, the images then combined (§3.1 process items 1-5).  Here
// the sub-cubes are blocks of kC^3 cells: a thread block copies one
// sub-cube's voxels (with a margin) from the bricks into shared memory, then
// marches, for every view of the launch, the samples of every ray that fall
// in it, and merges each ray's partial maximum into the image with an atomic
// maximum (the combining operator of MIP, which needs no visibility order).
// A voxel is read from HBM once per launch instead of once per view.
//
// Which sub-cube takes a sample.  Along each axis the sub-cube boundaries
// are planes x = c (c a multiple of kC); the first sample at or past such a
// plane in the ray's direction is k_c = ceil(((c - o) / d - t_entry) / step)
// (clamped to [0, K]), computed by the same instructions in both sub-cubes
// that share the plane, so the k-intervals of neighbouring sub-cubes meet
// exactly and every sample of a ray is taken by one sub-cube (per axis the
// planes cut [0, K) into intervals; a sample's sub-cube is the product of
// its three intervals).  An axis the ray is (nearly) parallel to assigns
// the sub-cube of the origin's cell.  k_c is the exact crossing up to
// rounding, so a sample lies within half a step of its sub-cube's box; the
// staged margin (cells c0 - 1 .. c0 + kC) covers it, and each sample is then
// computed exactly as the texture march computes it (position from the
// integer k, floors, fractions, eight corners clamped to the cube, the same
// interpolation), so the image and the sample count are vr_render's MIP bit
// for bit.
#include <cuda_fp16.h>

#include "vr_internal.h"
#include "vr_ray.cuh"

namespace vr {
namespace {

constexpr int kC = 32;                      // cells per sub-cube edge
constexpr int kE = kC + 3;                  // staged voxels per edge (cells c0 - 1 .. c0 + kC)
constexpr int kE2 = kE * kE;
constexpr int kStaged = kE * kE2;           // 42875 voxels: 171.5 KB as float
constexpr int kThreads = 1024;
constexpr unsigned kLastBase = kStaged - 1 - kE2 - kE - 1;   // largest corner-(0,0,0) index
constexpr float kParallel = 1e-20f;         // |d| below this: the axis is parallel

// One view's pixels that can reach the sub-cube: columns [x0, x0 + 8 npx),
// rows [y0, y1], in 8 x 4 packets; `first` is the view's first packet in the
// block's list.
struct Rect {
    int x0, y0, x1, y1, npx, first;
};

// Pixel rectangle of view c whose rays can meet the box [lo, hi] (positions,
// voxel units): the corners projected through the camera, with a two-pixel
// margin; the whole image when the box reaches behind a perspective eye or
// the camera's axes are degenerate.
__device__ Rect footprint(const MarchParams& P, const vr_camera& c, const float lo[3],
                          const float hi[3])
{
    // solve [fwd du dv] (a, b, c)^T = X - eye by the adjugate
    const float m00 = c.fwd[0], m01 = c.du[0], m02 = c.dv[0];
    const float m10 = c.fwd[1], m11 = c.du[1], m12 = c.dv[1];
    const float m20 = c.fwd[2], m21 = c.du[2], m22 = c.dv[2];
    const float i00 = m11 * m22 - m12 * m21, i01 = m02 * m21 - m01 * m22,
                i02 = m01 * m12 - m02 * m11;
    const float i10 = m12 * m20 - m10 * m22, i11 = m00 * m22 - m02 * m20,
                i12 = m02 * m10 - m00 * m12;
    const float i20 = m10 * m21 - m11 * m20, i21 = m01 * m20 - m00 * m21,
                i22 = m00 * m11 - m01 * m10;
    const float det = m00 * i00 + m01 * i10 + m02 * i20;
    Rect r;
    r.x0 = 0;
    r.y0 = 0;
    r.x1 = P.w - 1;
    r.y1 = P.h - 1;
    bool full = !(fabsf(det) > 0.0f) || !isfinite(det);
    float umin = INFINITY, umax = -INFINITY, vmin = INFINITY, vmax = -INFINITY;
    for (int i = 0; i < 8 && !full; ++i) {
        const float X0 = ((i & 1) ? hi[0] : lo[0]) - c.eye[0];
        const float X1 = ((i & 2) ? hi[1] : lo[1]) - c.eye[1];
        const float X2 = ((i & 4) ? hi[2] : lo[2]) - c.eye[2];
        const float a = (i00 * X0 + i01 * X1 + i02 * X2) / det;
        float u = (i10 * X0 + i11 * X1 + i12 * X2) / det;
        float v = (i20 * X0 + i21 * X1 + i22 * X2) / det;
        if (c.proj == VR_PERSP) {
            if (!(a > 0.0f)) {
                full = true;
                break;
            }
            u /= a;
            v /= a;
        }
        umin = fminf(umin, u);
        umax = fmaxf(umax, u);
        vmin = fminf(vmin, v);
        vmax = fmaxf(vmax, v);
    }
    if (!full) {
        // pixel px has u = px + 1/2 - w/2; clamp in float before converting
        const float bx = 0.5f * (float)P.w - 0.5f, by = 0.5f * (float)P.h - 0.5f;
        const float fw = (float)P.w, fh = (float)P.h;
        r.x0 = (int)fminf(fmaxf(floorf(umin + bx) - 2.0f, 0.0f), fw);
        r.x1 = (int)fminf(fmaxf(ceilf(umax + bx) + 2.0f, -1.0f), fw - 1.0f);
        r.y0 = (int)fminf(fmaxf(floorf(vmin + by) - 2.0f, 0.0f), fh);
        r.y1 = (int)fminf(fmaxf(ceilf(vmax + by) + 2.0f, -1.0f), fh - 1.0f);
        if (!(umin == umin) || !(umax == umax) || !(vmin == vmin) || !(vmax == vmax)) {
            r.x0 = 0;
            r.y0 = 0;
            r.x1 = P.w - 1;
            r.y1 = P.h - 1;
        }
    }
    return r;
}

// First sample at or past the plane at `c` on an axis (see the file comment).
__device__ __forceinline__ float plane_k(float c, float o, float inv_d, float te, float inv_step,
                                         float Kf)
{
    const float t = __fmul_rn(__fsub_rn(c, o), inv_d);
    const float q = __fmul_rn(__fsub_rn(t, te), inv_step);
    return ceilf(fminf(fmaxf(q, 0.0f), Kf));
}

// Narrow [ka, kb) to the samples of the sub-cube whose cells on this axis are
// [c0, c0 + kC) (the first sub-cube also takes cells below 0, the last those
// above, positions a rounding error outside the box).
__device__ __forceinline__ void axis_range(float o, float d, int c0, bool first, bool last,
                                           int n, float te, float inv_step, float Kf, float& ka,
                                           float& kb)
{
    if (fabsf(d) < kParallel) {
        // the cell of every sample is the origin's (d moves no position by a
        // representable amount); clamped to the cube's cells
        const int cell = min(max(__float2int_rd(o), 0), n - 2);
        if (cell < c0 || cell >= c0 + kC) kb = 0.0f;
        return;
    }
    const float inv_d = __frcp_rn(d);
    const float klo = first ? (d > 0.0f ? 0.0f : Kf)
                            : plane_k((float)c0, o, inv_d, te, inv_step, Kf);
    const float khi = last ? (d > 0.0f ? Kf : 0.0f)
                           : plane_k((float)(c0 + kC), o, inv_d, te, inv_step, Kf);
    if (d > 0.0f) {
        ka = fmaxf(ka, klo);
        kb = fminf(kb, khi);
    } else {
        ka = fmaxf(ka, khi);
        kb = fminf(kb, klo);
    }
}

__device__ __forceinline__ void atomic_max_float(float* a, float v)
{
    // IEEE order on the bit patterns: non-negative floats as signed integers
    // (max), negative ones as unsigned (min); -inf is the start value
    const int b = __float_as_int(v);
    if (b >= 0)
        atomicMax(reinterpret_cast<int*>(a), b);
    else
        atomicMin(reinterpret_cast<unsigned*>(a), (unsigned)b);
}

template <int DT>
__device__ __forceinline__ float load_staged(const MarchParams& P, int x, int y, int z)
{
    const VolumeGeom& g = P.g;
    const size_t brick = ((size_t)(z >> kBrickShift) * g.nby + (y >> kBrickShift)) * g.nbx +
                         (x >> kBrickShift);
    const size_t at = brick * kBrickVoxels + ((z & 31) << 10) + ((y & 31) << 5) + (x & 31);
    if constexpr (DT == VR_F32) return __ldg(static_cast<const float*>(P.bricks) + at);
    if constexpr (DT == VR_F16)
        return __half2float(__ldg(static_cast<const __half*>(P.bricks) + at));
    return (float)__ldg(static_cast<const signed char*>(P.bricks) + at);   // int8 code
}

template <int DT>
__global__ void __launch_bounds__(kThreads, 1)
    object_kernel(const __grid_constant__ MarchParams P, int k_max, int sx, int sy, int sz)
{
    extern __shared__ float4 s_dyn[];
    float* vox = reinterpret_cast<float*>(s_dyn);
    __shared__ Rect s_rect[kMaxViewsPerLaunch];
    __shared__ float2 s_dec[kE];
    __shared__ int s_next, s_total;
    __shared__ unsigned long long s_count;

    const int b = blockIdx.x;
    const int jx = b % sx, jy = (b / sx) % sy, jz = b / (sx * sy);
    const int c0x = jx * kC, c0y = jy * kC, c0z = jz * kC;
    const int nx = P.g.nx, ny = P.g.ny, nz = P.g.nz;

    // stage voxels c0 - 1 .. c0 + kC + 1 of each axis, clamped to the cube
    for (int i = threadIdx.x; i < kStaged; i += kThreads) {
        const int lz = i / kE2, rem = i - lz * kE2, ly = rem / kE, lx = rem - ly * kE;
        const int x = min(max(c0x - 1 + lx, 0), nx - 1);
        const int y = min(max(c0y - 1 + ly, 0), ny - 1);
        const int z = min(max(c0z - 1 + lz, 0), nz - 1);
        vox[i] = load_staged<DT>(P, x, y, z);
    }
    if constexpr (DT == VR_I8) {
        for (int i = threadIdx.x; i < kE; i += kThreads) {
            const int z = min(max(c0z - 1 + i, 0), nz - 1);
            s_dec[i] = make_float2(__ldg(P.scale + z), __ldg(P.offset + z));
        }
    }
    if (threadIdx.x < P.n_views) {
        const float lo[3] = {(float)(c0x - 1), (float)(c0y - 1), (float)(c0z - 1)};
        const float hi[3] = {(float)(c0x + kC + 1), (float)(c0y + kC + 1),
                             (float)(c0z + kC + 1)};
        s_rect[threadIdx.x] = footprint(P, P.cams[threadIdx.x], lo, hi);
    }
    if (threadIdx.x == 0) {
        s_next = 0;
        s_count = 0;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        int total = 0;
        for (int v = 0; v < P.n_views; ++v) {
            Rect& r = s_rect[v];
            r.npx = r.x1 >= r.x0 ? (r.x1 - r.x0) / 8 + 1 : 0;
            const int npy = r.y1 >= r.y0 ? (r.y1 - r.y0) / 4 + 1 : 0;
            r.first = total;
            total += r.npx * npy;
        }
        s_total = total;
    }
    __syncthreads();

    const int lane = threadIdx.x & 31;
    const bool first_x = jx == 0, last_x = jx == sx - 1;
    const bool first_y = jy == 0, last_y = jy == sy - 1;
    const bool first_z = jz == 0, last_z = jz == sz - 1;
    const float inv_step = __frcp_rn(P.step);
    // smem index of cell (ix, iy, iz) from the floor-shift bit patterns
    // (ix = bits - kFloorShiftBits; local = ix - (c0 - 1)), in wrapping
    // unsigned arithmetic
    const unsigned base = 0u - ((unsigned)(ray::kFloorShiftBits + c0z - 1) * kE +
                                (unsigned)(ray::kFloorShiftBits + c0y - 1)) * kE -
                          (unsigned)(ray::kFloorShiftBits + c0x - 1);
    unsigned long long count = 0;
    const int total = s_total;
    for (;;) {
        int pk = 0;
        if (lane == 0) pk = atomicAdd(&s_next, 1);
        pk = __shfl_sync(0xffffffffu, pk, 0);
        if (pk >= total) break;
        // the view: the last one whose first packet is at or before pk
        const unsigned m0 = __ballot_sync(0xffffffffu, lane < P.n_views && s_rect[lane].first <= pk);
        const unsigned m1 = __ballot_sync(0xffffffffu, lane + 32 < P.n_views &&
                                                           s_rect[lane + 32].first <= pk);
        const int view = m1 ? 63 - __clz(m1) : 31 - __clz(m0);
        const Rect& rc = s_rect[view];
        const int q = pk - rc.first, prow = q / rc.npx, pcol = q - prow * rc.npx;
        const int px = rc.x0 + pcol * 8 + (lane & 7), py = rc.y0 + prow * 4 + (lane >> 3);
        if (px > rc.x1 || py > rc.y1) continue;
        const ray::Ray r = ray::setup_ray(P, P.cams[view], px, py, k_max);
        if (r.K <= 0) continue;
        const float Kf = (float)r.K;
        float ka = 0.0f, kb = Kf;
        axis_range(r.ox, r.dx, c0x, first_x, last_x, nx, r.te, inv_step, Kf, ka, kb);
        axis_range(r.oy, r.dy, c0y, first_y, last_y, ny, r.te, inv_step, Kf, ka, kb);
        axis_range(r.oz, r.dz, c0z, first_z, last_z, nz, r.te, inv_step, Kf, ka, kb);
        if (!(ka < kb)) continue;
        float m = -INFINITY;
        for (float kf = ka; kf < kb; kf += 1.0f) {
            const float t = fmaf(kf, P.step, r.te);
            const float ppx = fmaf(t, r.dx, r.ox), ppy = fmaf(t, r.dy, r.oy),
                        ppz = fmaf(t, r.dz, r.oz);
            const float sx_ = __fadd_rd(ppx, ray::kFloorShift);
            const float sy_ = __fadd_rd(ppy, ray::kFloorShift);
            const float sz_ = __fadd_rd(ppz, ray::kFloorShift);
            ray::Geo g;
            g.fx = ppx - (sx_ - ray::kFloorShift);
            g.fy = ppy - (sy_ - ray::kFloorShift);
            g.fz = ppz - (sz_ - ray::kFloorShift);
            const unsigned at0 =
                ((unsigned)__float_as_int(sz_) * kE + (unsigned)__float_as_int(sy_)) * kE +
                (unsigned)__float_as_int(sx_) + base;
            ray::debug_ok(at0 <= kLastBase, 16);
            const unsigned at = min(at0, kLastBase);   // never needed (see above)
            // q = ((x0,y1), (x1,y1), (x1,y0), (x0,y0)) of planes z0 and z0 + 1
            const float4 q0 = make_float4(vox[at + kE], vox[at + kE + 1], vox[at + 1], vox[at]);
            const float4 q1 = make_float4(vox[at + kE2 + kE], vox[at + kE2 + kE + 1],
                                          vox[at + kE2 + 1], vox[at + kE2]);
            float s;
            if constexpr (DT == VR_I8) {
                const int lz = (int)(at / kE2);
                g.d0 = s_dec[lz];
                g.d1 = s_dec[lz + 1];
                s = ray::interp_t<VR_I8, true>(TexParams{}, q0, q1, g);
            } else {
                s = ray::interp(q0, q1, g);
            }
            m = fmaxf(m, s);
        }
        count += (unsigned long long)(kb - ka);
        if (m > -INFINITY) {
            const size_t pix = ((size_t)view * P.h + py) * P.w + px;
            if (ray::debug_ok(pix < (size_t)P.n_views * P.w * P.h, 1))
                atomic_max_float(P.out + pix, m);
        }
    }
    if (P.samples) {
        // one add per block
        for (int o = 16; o > 0; o >>= 1) count += __shfl_down_sync(0xffffffffu, count, o);
        if (lane == 0 && count) atomicAdd(&s_count, count);
        __syncthreads();
        if (threadIdx.x == 0 && s_count) atomicAdd(P.samples, s_count);
    }
}

template <int DT>
cudaError_t launch(const MarchParams& p, int k_max, cudaStream_t s)
{
    const int sx = (p.g.nx - 2) / kC + 1, sy = (p.g.ny - 2) / kC + 1, sz = (p.g.nz - 2) / kC + 1;
    const size_t smem = (size_t)kStaged * sizeof(float);
    static bool attr = false;   // set once per process (the value never changes)
    if (!attr) {
        cudaError_t e = cudaFuncSetAttribute(object_kernel<DT>,
                                             cudaFuncAttributeMaxDynamicSharedMemorySize,
                                             (int)smem);
        if (e != cudaSuccess) return e;
        attr = true;
    }
    object_kernel<DT><<<sx * sy * sz, kThreads, smem, s>>>(p, k_max, sx, sy, sz);
    return cudaGetLastError();
}

}  // namespace

cudaError_t launch_object(const MarchParams& p, int k_max, int dtype, cudaStream_t s)
{
    switch (dtype) {
    case VR_F32: return launch<VR_F32>(p, k_max, s);
    case VR_F16: return launch<VR_F16>(p, k_max, s);
    case VR_I8: return launch<VR_I8>(p, k_max, s);
    default: return cudaErrorInvalidValue;
    }
}

VR_DEBUG_ACCESSOR(debug_flags_object)

}  // namespace vr
