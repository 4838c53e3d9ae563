// vr_slab.cu -- the slab-staged ray-march kernel (the render hot path).
//
// Same rendering as vr_march.cu (paper §3.1 process item 3; definition in
// include/vr.h), but the eight-corner gather is served from shared memory:
//
//  * A block renders a 16 x 16 tile of rays (one thread per ray, warps of 8 x 4
//    neighbouring rays).  The tile takes as its principal axis a the largest
//    component of its central ray's direction; its rays advance monotonically
//    along a.
//  * The block walks the cube in slabs of S cells along a, in the direction of
//    travel.  For each slab it reduces, over its unfinished rays, the range of
//    the two other axes their samples can reach inside the slab (from the ray
//    equation at the slab's two bounding planes, widened by a margin), and
//    stages that window of the bricked cube -- S + 1 planes -- into shared
//    memory with cp.async: 16-byte copies along x when x is the window's
//    innermost axis, 4-byte copies when x is the principal axis.
//  * Each ray then takes its samples whose cell lies in the slab, reading the
//    corners from shared memory (a cell not entirely inside the staged window
//    -- the margin makes that rare -- is read from global memory), and stops
//    at the first sample of the next slab; the block moves on when every ray
//    has.  A ray reuses its last cell's corners while consecutive samples stay
//    in the same cell.
//  * Rays that do not advance along a with the tile, and any samples left
//    after the slab walk, are finished with global gathers.
//
// Sample positions are exactly those of vr_march.cu: t_k = fma(k, step,
// t_entry) from the integer k, p = fma(t_k, d, o) clamped to the box.  At a
// sample exactly on a far face (p = n - 1) the cell index here is n - 1 with
// weight 0 on a zero neighbour (vr_march.cu uses n - 2 with weight 1); both
// give the voxel's value.
#include <climits>

#include <cuda_fp16.h>

#include "vr_internal.h"

namespace vr {
namespace {

constexpr int kTile = 16;                  // 16 x 16 rays per block
constexpr int kThreads = kTile * kTile;
constexpr int kSmemHeader = VR_MAX_LUT * 16 + 64 + 128;   // table, reduction, corner rays

__device__ __forceinline__ float lerpf(float a, float b, float f) { return fmaf(f, b - a, a); }

__device__ __forceinline__ size_t brick_index(const VolumeGeom& g, int x, int y, int z)
{
    const size_t brick = ((size_t)(z >> kBrickShift) * g.nby + (y >> kBrickShift)) * g.nbx +
                         (x >> kBrickShift);
    return brick * kBrickVoxels + ((z & 31) << 10) + ((y & 31) << 5) + (x & 31);
}

// Voxel (x, y, z) >= 0 from global memory; zero beyond the cube.
__device__ __forceinline__ float voxel_global(const MarchParams& P, int x, int y, int z)
{
    if (x >= P.g.nx || y >= P.g.ny || z >= P.g.nz) return 0.0f;
    return __ldg(static_cast<const float*>(P.bricks) + brick_index(P.g, x, y, z));
}

// A staged box [x0, x0+ex) x [y0, y0+ey) x [z0, z0+ez) with element strides.
// A cell (its two corners per axis) is served from it iff 0 <= i - origin <
// extent - 1 on every axis; extents of 1 make every cell miss.
struct Window {
    int x0, y0, z0;
    int ex, ey, ez;
    int sx, sy, sz;
};

struct Ray {
    float ox, oy, oz, dx, dy, dz, te;
    int K, k;
    bool done;
    int cx, cy, cz;        // cached cell (-2: none)
    float c[8];            // its corners: bit 0 = +x, bit 1 = +y, bit 2 = +z
};

template <int MODE> struct Acc;
template <> struct Acc<VR_MIP> { float m = -INFINITY; };
template <> struct Acc<VR_SUM> { float m = 0.0f; };
template <> struct Acc<VR_COMPOSITE> { float r = 0.0f, g = 0.0f, b = 0.0f, A = 0.0f; };

__device__ __forceinline__ bool accumulate(const MarchParams&, const float4*, Acc<VR_MIP>& acc,
                                           float s)
{
    acc.m = fmaxf(acc.m, s);
    return false;
}

__device__ __forceinline__ bool accumulate(const MarchParams& P, const float4*, Acc<VR_SUM>& acc,
                                           float s)
{
    acc.m = fmaf(s, P.step, acc.m);
    return false;
}

__device__ __forceinline__ bool accumulate(const MarchParams& P, const float4* __restrict__ lut,
                                           Acc<VR_COMPOSITE>& acc, float s)
{
    if (!(s >= P.clip)) return false;
    const float x = fminf(fmaxf((s - P.v_lo) * P.lut_scale, 0.0f), P.lut_max);
    const int i = min((int)x, P.n_lut - 2);
    const float f = x - (float)i;
    const float4 a = lut[i], b = lut[i + 1];
    const float alpha = lerpf(a.w, b.w, f);
    const float wgt = (1.0f - acc.A) * alpha;
    acc.r = fmaf(wgt, lerpf(a.x, b.x, f), acc.r);
    acc.g = fmaf(wgt, lerpf(a.y, b.y, f), acc.g);
    acc.b = fmaf(wgt, lerpf(a.z, b.z, f), acc.b);
    acc.A += wgt;
    return acc.A >= P.term_alpha;
}

__device__ __forceinline__ void store(const MarchParams& P, size_t pix, const Acc<VR_MIP>& a)
{
    P.out[pix] = a.m;
}
__device__ __forceinline__ void store(const MarchParams& P, size_t pix, const Acc<VR_SUM>& a)
{
    P.out[pix] = a.m;
}
__device__ __forceinline__ void store(const MarchParams& P, size_t pix,
                                      const Acc<VR_COMPOSITE>& a)
{
    reinterpret_cast<float4*>(P.out)[pix] = make_float4(a.r, a.g, a.b, a.A);
}

// Camera -> ray -> box, exactly as in vr_march.cu.
__device__ __forceinline__ void setup(const MarchParams& P, const vr_camera& c, int px, int py,
                                      int k_max, Ray& r)
{
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
    if (!(nrm > 0.0f) || !isfinite(nrm)) return;
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
}

__device__ __forceinline__ float pick(float x, float y, float z, int a)
{
    return a == 0 ? x : (a == 1 ? y : z);
}

// Sample position of step k, clamped to the box.
__device__ __forceinline__ void position(const MarchParams& P, const Ray& r, int k, float& px,
                                         float& py, float& pz)
{
    const float t = fmaf((float)k, P.step, r.te);
    px = fminf(fmaxf(fmaf(t, r.dx, r.ox), 0.0f), P.hix);
    py = fminf(fmaxf(fmaf(t, r.dy, r.oy), 0.0f), P.hiy);
    pz = fminf(fmaxf(fmaf(t, r.dz, r.oz), 0.0f), P.hiz);
}

// March ray r through samples whose cell along axis a lies in [lo, hi)
// (lo = INT_MIN, hi = INT_MAX: all remaining samples).  Corners come from
// window w when the cell lies inside it.
template <int MODE>
__device__ __forceinline__ void march(const MarchParams& P, const float* __restrict__ win,
                                      const Window& w, const float4* __restrict__ lut, int a,
                                      int lo, int hi, Ray& r, Acc<MODE>& acc)
{
    while (r.k < r.K) {
        float px, py, pz;
        position(P, r, r.k, px, py, pz);
        const float flx = floorf(px), fly = floorf(py), flz = floorf(pz);
        const int ca = (int)pick(flx, fly, flz, a);
        if (ca < lo || ca >= hi) break;
        const int ix = (int)flx, iy = (int)fly, iz = (int)flz;
        if (ix != r.cx || iy != r.cy || iz != r.cz) {
            const unsigned rx = (unsigned)(ix - w.x0), ry = (unsigned)(iy - w.y0),
                           rz = (unsigned)(iz - w.z0);
            if (rx < (unsigned)(w.ex - 1) && ry < (unsigned)(w.ey - 1) &&
                rz < (unsigned)(w.ez - 1)) {
                const float* q = win + rx * w.sx + ry * w.sy + rz * w.sz;
                r.c[0] = q[0];
                r.c[1] = q[w.sx];
                r.c[2] = q[w.sy];
                r.c[3] = q[w.sx + w.sy];
                r.c[4] = q[w.sz];
                r.c[5] = q[w.sz + w.sx];
                r.c[6] = q[w.sz + w.sy];
                r.c[7] = q[w.sz + w.sx + w.sy];
            } else {
#pragma unroll
                for (int i = 0; i < 8; ++i)
                    r.c[i] = voxel_global(P, ix + (i & 1), iy + ((i >> 1) & 1), iz + (i >> 2));
            }
            r.cx = ix;
            r.cy = iy;
            r.cz = iz;
        }
        const float fx = px - flx, fy = py - fly, fz = pz - flz;
        const float y0z0 = lerpf(r.c[0], r.c[1], fx);
        const float y1z0 = lerpf(r.c[2], r.c[3], fx);
        const float y0z1 = lerpf(r.c[4], r.c[5], fx);
        const float y1z1 = lerpf(r.c[6], r.c[7], fx);
        const float s = lerpf(lerpf(y0z0, y1z0, fy), lerpf(y0z1, y1z1, fy), fz);
        ++r.k;
        if (accumulate(P, lut, acc, s)) {
            r.done = true;
            return;
        }
    }
    if (r.k >= r.K) r.done = true;
}

__device__ __forceinline__ void cp_async4(float* smem, const float* gmem)
{
    const unsigned s = (unsigned)__cvta_generic_to_shared(smem);
    asm volatile("cp.async.ca.shared.global [%0], [%1], 4;\n" ::"r"(s), "l"(gmem));
}

__device__ __forceinline__ void cp_async16(float* smem, const float* gmem)
{
    const unsigned s = (unsigned)__cvta_generic_to_shared(smem);
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(s), "l"(gmem));
}

__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;\n" ::); }
__device__ __forceinline__ void cp_async_wait_1() { asm volatile("cp.async.wait_group 1;\n" ::); }
__device__ __forceinline__ void cp_async_wait_all() { asm volatile("cp.async.wait_all;\n" ::); }

// Issue the copies that stage window w (all threads; completion is awaited
// by the caller).  Work items are flattened and split with float
// reciprocals, exact for the counts used here (< 2^16).  Voxels beyond the
// brick padding are written as zeros directly.
__device__ void stage(const MarchParams& P, float* __restrict__ win, const Window& w, int a)
{
    const float* base = static_cast<const float*>(P.bricks);
    const unsigned lim_x = P.g.nbx * kBrick, lim_y = P.g.nby * kBrick, lim_z = P.g.nbz * kBrick;
    const float inv_ey = 1.0f / (float)w.ey;
    if (a != 0) {
        // x innermost with unit stride (w.x0, w.ex multiples of 4): 16-byte chunks
        const int cpr = w.ex >> 2;
        const float inv_cpr = 1.0f / (float)cpr;
        const int n = cpr * w.ey * w.ez;
        for (int e = threadIdx.x; e < n; e += kThreads) {
            const int row = (int)(((float)e + 0.5f) * inv_cpr);
            const int cx = e - row * cpr;
            const int rz = (int)(((float)row + 0.5f) * inv_ey);
            const int ry = row - rz * w.ey;
            const int x = w.x0 + 4 * cx, y = w.y0 + ry, z = w.z0 + rz;
            float* dst = win + 4 * cx + ry * w.sy + rz * w.sz;
            if ((unsigned)x < lim_x && (unsigned)y < lim_y && (unsigned)z < lim_z) {
                cp_async16(dst, base + brick_index(P.g, x, y, z));
            } else {
                dst[0] = 0.0f;
                dst[1] = 0.0f;
                dst[2] = 0.0f;
                dst[3] = 0.0f;
            }
        }
    } else {
        // x is the principal axis (w.ex = S + 1 planes): 4-byte copies, with
        // neighbouring threads on neighbouring x
        const float inv_ex = 1.0f / (float)w.ex;
        const int n = w.ex * w.ey * w.ez;
        for (int e = threadIdx.x; e < n; e += kThreads) {
            const int row = (int)(((float)e + 0.5f) * inv_ex);
            const int rx = e - row * w.ex;
            const int rz = (int)(((float)row + 0.5f) * inv_ey);
            const int ry = row - rz * w.ey;
            const int x = w.x0 + rx, y = w.y0 + ry, z = w.z0 + rz;
            float* dst = win + rx * w.sx + ry * w.sy + rz * w.sz;
            if ((unsigned)x < lim_x && (unsigned)y < lim_y && (unsigned)z < lim_z)
                cp_async4(dst, base + brick_index(P.g, x, y, z));
            else
                *dst = 0.0f;
        }
    }
}

// Block-wide min of v0, v2 and max of v1, v3 (s_red[0..3]); all threads call.
__device__ __forceinline__ void block_minmax4(int* s_red, int& v0, int& v1, int& v2, int& v3)
{
    const int lane = threadIdx.x & 31;
    if (threadIdx.x < 4) s_red[threadIdx.x] = (threadIdx.x & 1) ? INT_MIN : INT_MAX;
    __syncthreads();
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        v0 = min(v0, __shfl_xor_sync(0xffffffffu, v0, o));
        v1 = max(v1, __shfl_xor_sync(0xffffffffu, v1, o));
        v2 = min(v2, __shfl_xor_sync(0xffffffffu, v2, o));
        v3 = max(v3, __shfl_xor_sync(0xffffffffu, v3, o));
    }
    if (lane == 0) {
        atomicMin(&s_red[0], v0);
        atomicMax(&s_red[1], v1);
        atomicMin(&s_red[2], v2);
        atomicMax(&s_red[3], v3);
    }
    __syncthreads();
    v0 = s_red[0];
    v1 = s_red[1];
    v2 = s_red[2];
    v3 = s_red[3];
}

// The four rays through the corner pixels of a tile: every ray of the tile
// lies in their convex hull, so the hull's section by a slab bounds every
// sample the tile takes in that slab.
struct Corners {
    float o[4][3];
    float d[4][3];
    float inv_da[4];
};

// Window of slab [s0, s0 + S) along a: S + 1 planes, and in b and c the
// bounding box of the corner rays between the slab's two planes (clamped to
// the box), widened by the margin and by one for the upper corner.
__device__ __forceinline__ void slab_window(const MarchParams& P, const SlabConfig& C,
                                            const Corners& K, int a, int b, int c, int s0,
                                            Window& w)
{
    const float hi_a = a == 0 ? P.hix : (a == 1 ? P.hiy : P.hiz);
    const float pa0 = fminf(fmaxf((float)s0, 0.0f), hi_a);
    const float pa1 = fminf(fmaxf((float)(s0 + C.S), 0.0f), hi_a);
    float bl = INFINITY, bh = -INFINITY, cl = INFINITY, ch = -INFINITY;
#pragma unroll
    for (int i = 0; i < 4; ++i) {
        const float t0 = (pa0 - K.o[i][a]) * K.inv_da[i];
        const float t1 = (pa1 - K.o[i][a]) * K.inv_da[i];
        const float b0 = fmaf(t0, K.d[i][b], K.o[i][b]), b1 = fmaf(t1, K.d[i][b], K.o[i][b]);
        const float c0 = fmaf(t0, K.d[i][c], K.o[i][c]), c1 = fmaf(t1, K.d[i][c], K.o[i][c]);
        bl = fminf(bl, fminf(b0, b1));
        bh = fmaxf(bh, fmaxf(b0, b1));
        cl = fminf(cl, fminf(c0, c1));
        ch = fmaxf(ch, fmaxf(c0, c1));
    }
    const int n_b = (b == 0) ? P.g.nx : P.g.ny;
    const int n_c = (c == 1) ? P.g.ny : P.g.nz;
    const float hb = (float)n_b, hc = (float)n_c;
    // clamp in float first (the hull may reach far outside the box)
    int bmin = (int)floorf(fminf(fmaxf(bl, 0.0f), hb)) - C.margin;
    int bmax = (int)floorf(fminf(fmaxf(bh, 0.0f), hb)) + 1 + C.margin;
    int cmin = (int)floorf(fminf(fmaxf(cl, 0.0f), hc)) - C.margin;
    int cmax = (int)floorf(fminf(fmaxf(ch, 0.0f), hc)) + 1 + C.margin;
    bmin = min(max(bmin, 0), n_b - 1);
    bmax = max(min(bmax, n_b), bmin + 1);
    cmin = min(max(cmin, 0), n_c - 1);
    cmax = max(min(cmax, n_c), cmin + 1);
    // shape within the buffer: S + 1 planes of eb x ec (rows of eb padded
    // to a multiple of 4 when x is innermost), trimmed to the budget
    const int ea = C.S + 1;
    int eb, ec = cmax - cmin + 1;
    int e3[3], o3[3], s3[3];
    if (a != 0) {            // [a][c][b], b = x innermost, 16-byte rows
        bmin &= ~3;
        eb = min((bmax - bmin + 4) & ~3, (C.win_elems / (2 * ea)) & ~3);
        ec = min(ec, C.win_elems / (ea * eb));
        s3[b] = 1;
        s3[c] = eb;
        s3[a] = eb * ec;
    } else {                 // [c][b][a], the x planes innermost
        eb = min(bmax - bmin + 1, C.win_elems / (2 * C.ea_pitch));
        ec = min(ec, C.win_elems / (C.ea_pitch * eb + 1));
        s3[a] = 1;
        s3[b] = C.ea_pitch;
        s3[c] = C.ea_pitch * eb + 1;
    }
    e3[a] = ea;
    o3[a] = s0;
    e3[b] = eb;
    o3[b] = bmin;
    e3[c] = ec;
    o3[c] = cmin;
    w.x0 = o3[0];
    w.y0 = o3[1];
    w.z0 = o3[2];
    w.ex = e3[0];
    w.ey = e3[1];
    w.ez = e3[2];
    w.sx = s3[0];
    w.sy = s3[1];
    w.sz = s3[2];
}

template <int MODE, bool COUNT>
__global__ void __launch_bounds__(kThreads, 2) slab_kernel(const __grid_constant__ MarchParams P,
                                                           const SlabConfig C)
{
    extern __shared__ __align__(16) unsigned char smem_raw[];
    float4* s_lut = reinterpret_cast<float4*>(smem_raw);
    int* s_red = reinterpret_cast<int*>(smem_raw + VR_MAX_LUT * 16);
    Corners* s_k = reinterpret_cast<Corners*>(smem_raw + VR_MAX_LUT * 16 + 64);
    float* s_win[2] = {reinterpret_cast<float*>(smem_raw + kSmemHeader),
                       reinterpret_cast<float*>(smem_raw + kSmemHeader) + C.win_elems};

    if (MODE == VR_COMPOSITE)
        for (int i = threadIdx.x; i < P.n_lut; i += kThreads) s_lut[i] = P.lut[i];

    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int tx0 = blockIdx.x * kTile, ty0 = blockIdx.y * kTile;
    const int px = tx0 + (warp & 1) * 8 + (lane & 7);
    const int py = ty0 + (warp >> 1) * 4 + (lane >> 3);
    const int view = blockIdx.z;
    const bool valid = px < P.w && py < P.h;
    const vr_camera& cam = P.cams[view];

    Ray r;
    r.K = 0;
    r.te = 0.0f;
    r.ox = r.oy = r.oz = r.dx = r.dy = r.dz = 0.0f;
    if (valid) setup(P, cam, px, py, C.k_max, r);
    r.k = 0;
    r.done = (r.K == 0);
    r.cx = r.cy = r.cz = -2;

    // principal axis and direction of travel, from the tile's central ray
    int a;
    float sgn;
    {
        float d0, d1, d2;
        if (cam.proj == VR_ORTHO) {
            d0 = cam.fwd[0];
            d1 = cam.fwd[1];
            d2 = cam.fwd[2];
        } else {
            const float u = (float)(tx0 + kTile / 2) - 0.5f * (float)P.w;
            const float v = (float)(ty0 + kTile / 2) - 0.5f * (float)P.h;
            d0 = fmaf(v, cam.dv[0], fmaf(u, cam.du[0], cam.fwd[0]));
            d1 = fmaf(v, cam.dv[1], fmaf(u, cam.du[1], cam.fwd[1]));
            d2 = fmaf(v, cam.dv[2], fmaf(u, cam.du[2], cam.fwd[2]));
        }
        // slab along y or z when the ray advances well along one of them, so
        // that x (the brick rows) stays the window's innermost axis and the
        // window is staged with 16-byte copies; along x only otherwise
        const float nrm = sqrtf(d0 * d0 + d1 * d1 + d2 * d2);
        const float a1 = fabsf(d1), a2 = fabsf(d2);
        a = (fmaxf(a1, a2) >= C.min_axis * nrm) ? (a1 >= a2 ? 1 : 2) : 0;
        sgn = pick(d0, d1, d2, a) >= 0.0f ? 1.0f : -1.0f;
    }
    const int b = (a == 0) ? 1 : 0;     // the window's innermost axis
    const int c = (a == 2) ? 1 : 2;

    // corner rays of the tile (clamped to the image)
    if (threadIdx.x < 4) {
        Ray q;
        const int cxp = (threadIdx.x & 1) ? min(tx0 + kTile - 1, P.w - 1) : tx0;
        const int cyp = (threadIdx.x & 2) ? min(ty0 + kTile - 1, P.h - 1) : ty0;
        setup(P, cam, cxp, cyp, C.k_max, q);
        const int i = threadIdx.x;
        s_k->o[i][0] = q.ox; s_k->o[i][1] = q.oy; s_k->o[i][2] = q.oz;
        s_k->d[i][0] = q.dx; s_k->d[i][1] = q.dy; s_k->d[i][2] = q.dz;
        const float da = pick(q.dx, q.dy, q.dz, a);
        s_k->inv_da[i] = (da * sgn > 0.5f * C.min_axis) ? 1.0f / da : 0.0f;
    }

    // range of cells along a that the block's rays visit
    const float da_r = pick(r.dx, r.dy, r.dz, a);
    int lo_cell = INT_MAX, hi_cell = INT_MIN, bad = INT_MAX, u1 = INT_MIN;
    if (!r.done) {
        float px0, py0, pz0, px1, py1, pz1;
        position(P, r, 0, px0, py0, pz0);
        position(P, r, r.K - 1, px1, py1, pz1);
        const int c0 = (int)floorf(pick(px0, py0, pz0, a));
        const int c1 = (int)floorf(pick(px1, py1, pz1, a));
        lo_cell = min(c0, c1);
        hi_cell = max(c0, c1);
    }
    if (threadIdx.x < 4 && s_k->inv_da[threadIdx.x] == 0.0f) bad = 0;   // tile not monotone
    block_minmax4(s_red, lo_cell, hi_cell, bad, u1);
    const Corners K = *s_k;
    const bool tile_ok = bad != 0 && hi_cell >= lo_cell;
    const bool slab_ray = tile_ok && !r.done && da_r * sgn > 0.0f;
    const int n_slabs = tile_ok ? (hi_cell - lo_cell) / C.S + 1 : 0;

    Acc<MODE> acc;
    Window w_cur, w_next;
    if (n_slabs > 0) {
        const int s0 = (sgn > 0.0f) ? lo_cell : hi_cell - C.S + 1;
        slab_window(P, C, K, a, b, c, s0, w_cur);
        stage(P, s_win[0], w_cur, a);
        cp_async_commit();
    }
    for (int j = 0; j < n_slabs; ++j) {
        const int s0 = (sgn > 0.0f) ? lo_cell + j * C.S : hi_cell - (j + 1) * C.S + 1;
        if (j + 1 < n_slabs) {
            // prefetch the next slab into the other buffer
            const int s1 = (sgn > 0.0f) ? s0 + C.S : s0 - C.S;
            slab_window(P, C, K, a, b, c, s1, w_next);
            stage(P, s_win[(j + 1) & 1], w_next, a);
            cp_async_commit();
            cp_async_wait_1();
        } else {
            cp_async_wait_all();
        }
        __syncthreads();
        if (slab_ray && !r.done)
            march<MODE>(P, s_win[j & 1], w_cur, s_lut, a, s0, s0 + C.S, r, acc);
        // buffer j & 1 is restaged at j + 2: every ray must be done with it
        if (!__syncthreads_or(slab_ray && !r.done)) break;
        w_cur = w_next;
    }
    cp_async_wait_all();

    // rays outside the slab scheme, and samples the slab walk left over
    if (valid && !r.done) {
        Window none;
        none.x0 = none.y0 = none.z0 = 0;
        none.ex = none.ey = none.ez = 1;
        none.sx = none.sy = none.sz = 0;
        march<MODE>(P, s_win[0], none, s_lut, a, INT_MIN, INT_MAX, r, acc);
    }

    if (valid) store(P, ((size_t)view * P.h + py) * P.w + px, acc);
    if (COUNT) {
        const unsigned cnt = valid ? (unsigned)r.k : 0u;
        const unsigned tot = __reduce_add_sync(0xffffffffu, cnt);
        if (lane == 0 && tot) atomicAdd(P.samples, (unsigned long long)tot);
    }
}

template <int MODE, bool COUNT>
cudaError_t launch_one(const MarchParams& p, const SlabConfig& c, cudaStream_t s)
{
    dim3 grid((unsigned)((p.w + kTile - 1) / kTile), (unsigned)((p.h + kTile - 1) / kTile),
              (unsigned)p.n_views);
    cudaError_t e = cudaFuncSetAttribute(slab_kernel<MODE, COUNT>,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)c.smem_bytes);
    if (e != cudaSuccess) return e;
    slab_kernel<MODE, COUNT><<<grid, kThreads, c.smem_bytes, s>>>(p, c);
    return cudaGetLastError();
}

template <int MODE>
cudaError_t launch_m(const MarchParams& p, const SlabConfig& c, cudaStream_t s)
{
    return p.samples ? launch_one<MODE, true>(p, c, s) : launch_one<MODE, false>(p, c, s);
}

}  // namespace

size_t slab_window_elems(const SlabConfig& c)
{
    return ((size_t)c.win_elems + 3) & ~(size_t)3;   // keeps the second buffer 16-byte aligned
}

size_t slab_smem_bytes(const SlabConfig& c)
{
    return kSmemHeader + 2 * 4 * slab_window_elems(c);   // two windows: double buffering
}

cudaError_t launch_slab(const MarchParams& p, const SlabConfig& c, int mode, cudaStream_t s)
{
    switch (mode) {
    case VR_MIP: return launch_m<VR_MIP>(p, c, s);
    case VR_COMPOSITE: return launch_m<VR_COMPOSITE>(p, c, s);
    default: return launch_m<VR_SUM>(p, c, s);
    }
}

}  // namespace vr
