// vr_ray.cuh -- the per-ray march shared by the render kernels (device code).
//
// One ray per thread (paper §3.1 process item 3; definition in include/vr.h):
// camera -> ray -> box -> K samples at t_entry + k*step -> trilinear value ->
// MIP / SUM / clipped table + front-to-back compositing with termination.
// Two ways to fetch a cell's eight corners:
//   * texture storage: one unfiltered four-texel gather (tld4) per plane of
//     a layered 2-D texture (one layer per frequency plane), pipelined one
//     sample ahead, with the last cell's corners reused;
//   * brick storage: eight read-only loads from 32^3 bricks.
// The functions are templated on the parameter record (PP: image, volume and
// transfer scalars) so the per-view kernel and the batched kernel share them.
#pragma once

#include <cuda_fp16.h>

#include "vr_internal.h"

namespace vr {
namespace ray {

// ---- the checked build (compiled with VR_DEBUG) ----
// Kernels test the indices they compute against the buffers they address;
// a failed test records its bit in a device word of the translation unit and
// the access is skipped (no trap, no fault): vr_debug_status reads and
// clears the words.  Bits: 1 an output pixel outside the image set, 2 a
// brick address outside the brick buffer, 4 a partial image index outside
// the integration's input, 8 a batched tile outside its request, 16 an
// object-order sample outside its staged sub-cube.  Without
// VR_DEBUG the tests compile to nothing.
#ifdef VR_DEBUG
static __device__ unsigned g_debug_flags;
__device__ __forceinline__ bool debug_ok(bool cond, unsigned bit)
{
    if (!cond) atomicOr(&g_debug_flags, bit);
    return cond;
}
#define VR_DEBUG_ACCESSOR(name)                                                   \
    unsigned name(bool clear)                                                     \
    {                                                                             \
        unsigned v = 0;                                                           \
        if (cudaMemcpyFromSymbol(&v, ray::g_debug_flags, sizeof v) != cudaSuccess) \
            v = 0x80000000u;                                                      \
        if (clear) {                                                              \
            const unsigned zero = 0;                                              \
            cudaMemcpyToSymbol(ray::g_debug_flags, &zero, sizeof zero);           \
        }                                                                         \
        return v;                                                                 \
    }
#else
__device__ __forceinline__ constexpr bool debug_ok(bool, unsigned) { return true; }
#define VR_DEBUG_ACCESSOR(name) \
    unsigned name(bool) { return 0; }
#endif

__device__ __forceinline__ float lerpf(float a, float b, float f) { return fmaf(f, b - a, a); }

// Two floats in one 64-bit register pair, for the packed FP32 instructions
// (f32x2: the same IEEE operation on both halves).
__device__ __forceinline__ unsigned long long pack2(float lo, float hi)
{
    unsigned long long r;
    asm("mov.b64 %0, {%1, %2};" : "=l"(r) : "f"(lo), "f"(hi));
    return r;
}

__device__ __forceinline__ float2 unpack2(unsigned long long r)
{
    float2 f;
    asm("mov.b64 {%0, %1}, %2;" : "=f"(f.x), "=f"(f.y) : "l"(r));
    return f;
}

// a - b on both halves, rounded to nearest.
__device__ __forceinline__ unsigned long long sub2(unsigned long long a, unsigned long long b)
{
    unsigned long long d;
    asm("sub.rn.f32x2 %0, %1, %2;" : "=l"(d) : "l"(a), "l"(b));
    return d;
}

// fma(a, b, c) on both halves.
__device__ __forceinline__ unsigned long long fma2(unsigned long long a, unsigned long long b,
                                                   unsigned long long c)
{
    unsigned long long d;
    asm("fma.rn.f32x2 %0, %1, %2, %3;" : "=l"(d) : "l"(a), "l"(b), "l"(c));
    return d;
}

// lerpf on both halves: fma(f, b - a, a), rounded as lerpf.
__device__ __forceinline__ unsigned long long lerp2(unsigned long long a, unsigned long long b,
                                                    unsigned long long f)
{
    unsigned long long d, r;
    asm("sub.rn.f32x2 %0, %1, %2;" : "=l"(d) : "l"(b), "l"(a));
    asm("fma.rn.f32x2 %0, %1, %2, %3;" : "=l"(r) : "l"(f), "l"(d), "l"(a));
    return r;
}


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

// The height component of a pixel's ray direction before normalisation,
// computed as setup_ray computes it: the ray goes up (or is level) exactly
// when it is >= 0, as setup_ray's r.dz.
__device__ __forceinline__ float ray_dz_raw(const vr_camera& c, int w, int h, int px, int py)
{
    if (c.proj == VR_ORTHO) return c.fwd[2];
    const float u = ((float)px + 0.5f) - 0.5f * (float)w;
    const float v = ((float)py + 0.5f) - 0.5f * (float)h;
    return fmaf(v, c.dv[2], fmaf(u, c.du[2], c.fwd[2]));
}

// Camera -> ray -> box -> sample count K (0 for a miss or a degenerate
// direction).  PP supplies w, h, hix, hiy, hiz and step.
template <typename PP>
__device__ __forceinline__ Ray setup_ray(const PP& P, const vr_camera& c, int px, int py,
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

__device__ __forceinline__ uint4 gather_u32(cudaTextureObject_t t, int layer, float x, float y)
{
    uint4 r;
    asm volatile("tld4.r.a2d.v4.u32.f32 {%0, %1, %2, %3}, [%4, {%5, %6, %7, %7}];"
                 : "=r"(r.x), "=r"(r.y), "=r"(r.z), "=r"(r.w)
                 : "l"(t), "r"(layer), "f"(x), "f"(y));
    return r;
}

__device__ __forceinline__ float half_bits(unsigned b)
{
    return __half2float(__ushort_as_half((unsigned short)(b & 0xffffu)));
}

// int8 pair texels hold each code q as the byte q + 128 (the fill flips its
// sign bit).  A byte permute places that byte under the exponent of 2^23, so
// the float is 2^23 + q + 128 exactly, and subtracting 2^23 + 128 leaves q
// exactly: the value (float)q from full-rate instructions instead of a
// conversion (interp_t; 1024^3 int8 pair, 32 views at 1080p: MIP 50.7 ->
// 43.9 ms).
constexpr float kCodeBias = 8388736.0f;   // 2^23 + 128

// Texture slices.  Plain formats: slice s holds plane s - 1, and slices 0
// and nz + 1 repeat planes 0 and nz - 1.  Pair formats: slice s holds the
// cell between planes s - 1 and s (clamped to [0, nz - 1]), s in [0, nz].
// A sample at height pz therefore reads slices floor(pz) + 1 (and + 2),
// with no clamping for positions a rounding error outside the z faces: the
// repeated edge planes give the edge value exactly.
//
// Layer and row offset of slice z.  Unstacked (a layer per slice): layer z,
// rows as stored.  Stacked: 2^shift slices per layer, slice z at sub-slice
// z & (2^shift - 1) of layer z >> shift, whose ny data rows start at row
// sub * pitch + 1 (rows sub * pitch and sub * pitch + ny + 1 copy its first
// and last rows, so a gather one row outside the data reads the edge row as
// the texture's clamp addressing does for an unstacked layer).
// Returns the layer; `yt` is the gather's y coordinate y in that layer.
template <bool STACK, typename TT>
__device__ __forceinline__ int plane_layer(const TT& T, int z, float y, float& yt)
{
    if (!STACK) {
        yt = y;
        return z;
    }
    yt = y + (float)((z & ((1 << T.stack_shift) - 1)) * T.stack_pitch + 1);
    return z >> T.stack_shift;
}

// The two planes of the cell at slice z (planes z - 1 and z, see above)
// whose x/y corner is texel (x-1, y-1).  Pair formats: one gather of slice z
// holds both planes.
template <int DT, bool STACK, typename TT>
__device__ __forceinline__ void cell(const TT& T, cudaTextureObject_t t0, int z, float x,
                                     float y, float4& q0, float4& q1)
{
    float yt;
    const int l = plane_layer<STACK>(T, z, y, yt);
    if constexpr (DT == kF16Pair || DT == kI8Pair) {
        // the packed texels as they are (their bits carried in q0; q1 unused):
        // unpacked when the sample is interpolated (interp_t), not when the
        // gather returns
        const uint4 p = gather_u32(t0, l, x, yt);
        q0 = make_float4(__uint_as_float(p.x), __uint_as_float(p.y), __uint_as_float(p.z),
                         __uint_as_float(p.w));
        q1 = q0;
    } else {
        float yt1;
        const int l1 = plane_layer<STACK>(T, z + 1, y, yt1);
        q0 = gather<DT>(t0, l, x, yt);           // int8: codes (see interp_t)
        q1 = gather<DT>(t0, l1, x, yt1);
    }
}

// Corners of the cell of sample geometry `n` given the cell `c` whose corners
// (c0, c1) are held.  Pair formats fetch the cell in one gather, every
// sample.  Plain formats fetch the lower and
// the upper plane in two gather slots that every lane of a warp shares, each
// skipped by the lanes that hold that plane already (the lower one when z
// rose by one, the upper one when z fell by one): whatever mix of moves the
// lanes make, a warp issues at most two gathers per sample.
template <int DT, bool STACK, bool KEEP_PAIR, typename TT, typename G>
__device__ __forceinline__ void next_cell(const TT& T, cudaTextureObject_t t0, const G& c,
                                          const float4& c0, const float4& c1, const G& n,
                                          float4& n0, float4& n1)
{
    if constexpr (DT == kF16Pair || DT == kI8Pair) {
        // the single-view kernels gather every sample, even in the same cell:
        // measured faster than testing for a change of cell and keeping the
        // held texels (1024^3 FP16, 32 views at 1080p: MIP 57.6 -> 44.5 ms,
        // composite 59.4 -> 48.9 ms), the test and selects costing more issue
        // slots than the gather.  The batched kernel, short of registers at
        // six blocks per SM, keeps them (KEEP_PAIR: 53.8 -> 49.1 ms on the
        // batched workload).  Plain formats keep their planes either way
        // (two gathers a sample measured slower than the slot test).
        if (KEEP_PAIR && n.gx == c.gx && n.gy == c.gy && n.iz == c.iz) {
            n0 = c0;
            n1 = c1;
        } else {
            cell<DT, STACK>(T, t0, n.iz, n.gx, n.gy, n0, n1);
        }
    } else {
        const bool xy = n.gx == c.gx && n.gy == c.gy;
        const int dz = n.iz - c.iz;
        // lower plane: held as c0 (same cell) or c1 (z rose by one); upper
        // plane: held as c1 (same cell) or c0 (z fell by one)
        const bool keep0 = xy && (dz == 0 || dz == 1);
        const bool keep1 = xy && (dz == 0 || dz == -1);
        float yt;
        if (keep0) {
            n0 = dz == 0 ? c0 : c1;
        } else {
            const int l = plane_layer<STACK>(T, n.iz, n.gy, yt);
            n0 = gather<DT>(t0, l, n.gx, yt);
        }
        if (keep1) {
            n1 = dz == 0 ? c1 : c0;
        } else {
            const int l = plane_layer<STACK>(T, n.iz + 1, n.gy, yt);
            n1 = gather<DT>(t0, l, n.gx, yt);
        }
    }
}

// floor(v) as an integer for |v| < 2^22 with one full-rate add (no
// float-to-int conversion): s = v + 1.5 * 2^23 rounded toward -infinity is
// floor(v) + 1.5 * 2^23 exactly, the float spacing in [2^23, 2^24) being 1,
// so s's low mantissa bits hold floor(v) (IEEE 754 binary32), and s - 1.5 *
// 2^23 is floor(v) as a float, exactly.  Sample positions stay within a
// voxel or so of the box, and cube edges are at most 2^20.
constexpr float kFloorShift = 0x1.8p23f;
constexpr int kFloorShiftBits = 0x4B400000;

__device__ __forceinline__ int floor_small(float v)
{
    return __float_as_int(__fadd_rd(v, kFloorShift)) - kFloorShiftBits;
}

// Per-sample geometry: the gather coordinates of the cell and the weights.
// Nothing is clamped to the box: a position just outside an x or y face (by
// rounding) has both its corners clamped to the edge texel by the texture
// unit, and one just outside a z face reads a repeated edge plane, which
// gives the edge value exactly as clamping the position would.
struct Geo {
    float gx, gy;     // gather coordinates (cell corner + 1)
    float fx, fy, fz;
    int iz;           // texture slice of the cell's lower plane (cell + 1)
    float2 d0, d1;    // plain int8: the decode records of slices iz, iz + 1;
                      // int8 pair: the planes' scales, then their offsets
};

template <typename PP>
__device__ __forceinline__ Geo geo(const PP& P, const Ray& r, float kf)
{
    Geo g;
    const float t = fmaf(kf, P.step, r.te);
    const float px = fmaf(t, r.dx, r.ox), py = fmaf(t, r.dy, r.oy), pz = fmaf(t, r.dz, r.oz);
    const float flx = floorf(px), fly = floorf(py);
    // the height's floor both as a float and as the slice index, from one
    // full-rate add (no float-to-int conversion; see floor_small)
    const float sz = __fadd_rd(pz, kFloorShift);
    const float flz = sz - kFloorShift;
    g.gx = flx + 1.0f;
    g.gy = fly + 1.0f;
    g.fx = px - flx;
    g.fy = py - fly;
    g.fz = pz - flz;
    g.iz = __float_as_int(sz) - (kFloorShiftBits - 1);
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

// int8: fetch the sample's decode records (plain: slices g.iz and g.iz + 1;
// pair: the one record of slice g.iz) along with its geometry, a step before
// they are used.
template <int DT, typename TT>
__device__ __forceinline__ void fetch_dec(const TT& T, Geo& g)
{
    if constexpr (DT == VR_I8) {
        g.d0 = __ldg(static_cast<const float2*>(T.dec) + g.iz);   // {scale, offset}
        g.d1 = __ldg(static_cast<const float2*>(T.dec) + g.iz + 1);
    } else if constexpr (DT == kI8Pair) {
        const float4 d = __ldg(static_cast<const float4*>(T.dec) + g.iz);   // both planes
        g.d0 = make_float2(d.x, d.y);   // the planes' scales
        g.d1 = make_float2(d.z, d.w);   // and offsets
    }
}

// interp for a texel format: int8 texels (plain and pair) are codes, so each plane's
// bilinear value of the codes is decoded with that plane's scale and offset
// (decoding is affine and the bilinear weights sum to one, so this is the
// interpolation of the decoded corners up to rounding), from the records of
// the cell's slices (g.iz, g.iz + 1: planes g.iz - 1 and g.iz, clamped):
// HELD, fetched with the geometry (fetch_dec, the marches over every sample);
// otherwise read here (the lockstep marches, whose registers are spoken
// for).  Two decodes a sample, applied when the sample is interpolated
// rather than when its gathers return, so no decode waits for a gather in
// flight; the records and the arithmetic are the same either way.
template <int DT, bool HELD, typename TT>
__device__ __forceinline__ float interp_t(const TT& T, const float4& q0, const float4& q1,
                                          const Geo& g)
{
    if constexpr (DT == kF16Pair) {
        // q0 carries the packed texels: plane g.iz - 1 in the low halves
        const unsigned px = __float_as_uint(q0.x), py = __float_as_uint(q0.y),
                       pz = __float_as_uint(q0.z), pw = __float_as_uint(q0.w);
        return interp(make_float4(half_bits(px), half_bits(py), half_bits(pz), half_bits(pw)),
                      make_float4(half_bits(px >> 16), half_bits(py >> 16), half_bits(pz >> 16),
                                  half_bits(pw >> 16)),
                      g);
    } else if constexpr (DT != VR_I8 && DT != kI8Pair) {
        return interp(q0, q1, g);
    } else if constexpr (DT == kI8Pair) {
        // both planes side by side in register pairs: each texel's two codes
        // unpacked by one packed subtraction (code_lo / code_hi), both
        // planes' bilinear lerps and decodes in packed instructions (the
        // same IEEE operations, in the same order, as the plain int8 path:
        // images identical)
        float2 sc, of;                       // the two planes' scales and offsets
        if constexpr (HELD) {
            sc = g.d0;
            of = g.d1;
        } else {
            const float4 d = __ldg(static_cast<const float4*>(T.dec) + g.iz);
            sc = make_float2(d.x, d.y);
            of = make_float2(d.z, d.w);
        }
        auto planes = [](float t) {          // q of plane g.iz - 1, q of plane g.iz
            const unsigned w = __float_as_uint(t);
            return sub2(pack2(__uint_as_float(__byte_perm(w, 0x4b000000u, 0x7540)),
                              __uint_as_float(__byte_perm(w, 0x4b000000u, 0x7541))),
                        pack2(kCodeBias, kCodeBias));
        };
        const unsigned long long fx = pack2(g.fx, g.fx), fy = pack2(g.fy, g.fy);
        const unsigned long long y0 = lerp2(planes(q0.w), planes(q0.z), fx);
        const unsigned long long y1 = lerp2(planes(q0.x), planes(q0.y), fx);
        const float2 v = unpack2(fma2(lerp2(y0, y1, fy), pack2(sc.x, sc.y), pack2(of.x, of.y)));
        return lerpf(v.x, v.y, g.fz);
    } else {                                  // plain int8: the two planes' codes
        float2 d0, d1;
        if constexpr (HELD) {
            d0 = g.d0;
            d1 = g.d1;
        } else {
            d0 = __ldg(static_cast<const float2*>(T.dec) + g.iz);   // {scale, offset}
            d1 = __ldg(static_cast<const float2*>(T.dec) + g.iz + 1);
        }
        const float b0 = lerpf(lerpf(q0.w, q0.z, g.fx), lerpf(q0.x, q0.y, g.fx), g.fy);
        const float b1 = lerpf(lerpf(q1.w, q1.z, g.fx), lerpf(q1.x, q1.y, g.fx), g.fy);
        return lerpf(fmaf(b0, d0.x, d0.y), fmaf(b1, d1.x, d1.y), g.fz);
    }
}

// Accumulate one sample; returns true when the ray terminates.
template <int MODE>
struct Acc {
    float r = 0.0f, g = 0.0f, b = 0.0f, A = 0.0f;
    float m = (MODE == VR_MIP) ? -INFINITY : 0.0f;

    template <typename PP>
    __device__ __forceinline__ bool add(const PP& P, const float4* __restrict__ lut, float s)
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

    // Skipping (march_win, COMPOSITE): may the sample whose
    // macrocell mask is `rec` and whose cell is bit `bit` of it be visible?
    __device__ __forceinline__ bool need(unsigned long long rec, int bit) const
    {
        return (rec >> bit) & 1ull;
    }
};

// ---- empty-space skipping ----
// The macrocell of sample kf and its cell's bit there, from the gather
// coordinates (cell + 1 on every axis: in [0, n] for positions inside the box
// up to rounding).  The index is clamped to the mask array: the look-ahead
// samples past a ray's end, and positions of cameras so far away that
// rounding moves them by a voxel, may lie outside, and their bits are never
// used.  (A function rather than a lambda, so that it is inlined in every
// kernel that marches with masks, the batched one included.)
// z_base: the first plane of a part volume (its masks cover its own planes).
template <typename PP>
__device__ __forceinline__ int mask_cell(const PP& P, const Ray& r, float kf, int& bit,
                                         int z_base = 0)
{
    const float t = fmaf(kf, P.step, r.te);
    const int x = floor_small(fmaf(t, r.dx, r.ox)) + 1;
    const int y = floor_small(fmaf(t, r.dy, r.oy)) + 1;
    const int z = floor_small(fmaf(t, r.dz, r.oz)) + 1 - z_base;
    bit = (x & 3) | ((y & 3) << 2) | ((z & 3) << 4);
    const int i = ((z >> kMacroShift) * P.mny + (y >> kMacroShift)) * P.mnx + (x >> kMacroShift);
    return (int)min((unsigned)i, (unsigned)P.mlast);
}

// march_tex with empty-space skipping in windows (COMPOSITE): the warp's
// lanes scan kWin samples in lockstep -- each step only the sample's cell,
// its mask word and bit, setting the step's bit in the lane's window mask
// when the clip can leave the sample visible -- and then evaluate the
// window's marked samples in order, lowest first, every lane taking its
// next one in the same round: the rare visible samples of a noise ray are
// evaluated together with the other lanes' instead of each in a lockstep
// step of its own (1024^3, 32 views at 1080p: 44.5 -> 37.3 ms against the
// lockstep march that tested and evaluated sample by sample).  Within a
// round the gathers of a lane's next sample are issued before its current
// one is interpolated.  Samples [k0, k1) are composited in increasing order
// with march_tex's arithmetic, so the result and the sample count (the
// samples stepped until the ray stops) are march_tex's.  PART: the volume
// holds a part of the cube starting at plane P.slice_base (texture slices
// and mask macrocells are the part's own).  All lanes of the calling warp
// that have samples must call it together (warp votes).
constexpr int kWin = 32;

template <int DT, int MODE, bool STACK, bool PART, typename PP, typename TT>
__device__ __forceinline__ int march_win(const PP& P, const TT& T, const float4* __restrict__ lut,
                                         const Ray& r, Acc<MODE>& acc, int k0, int k1)
{
    static_assert(MODE == VR_COMPOSITE, "skipping is for compositing");
    const unsigned lanes = __activemask();
    const cudaTextureObject_t t0 = T.tex;
    const int z_base = PART ? P.slice_base : 0;
    int stop = k1;                     // the samples stepped end here (k1 unless the ray stops)
    bool live = k0 < k1;
    for (int ws = k0; __any_sync(lanes, live); ws += kWin) {
        // scan: one bit per sample of the window that the clip can leave visible
        unsigned bits = 0;
        if (live) {
            const int n = min(kWin, k1 - ws);
            // sample ws + j is bit 31 - j, shifted in from the bottom; the
            // sample index stepped as a float (exact below 2^24), every step's
            // bit taken without a test and the steps past the ray's end
            // cleared once after the loop (1024^3, 32 views at 1080p: 37.4 ->
            // 32.4 ms against a conversion, a test of j < n and a shift by j
            // per step)
            float kj = (float)ws;
#pragma unroll 4
            for (int j = 0; j < kWin; ++j) {
                int bit;
                const int m = mask_cell(P, r, kj, bit, z_base);
                const unsigned long long rec = __ldg(P.mask + m);
                bits = bits * 2u + (unsigned)((rec >> bit) & 1ull);
                kj += 1.0f;
            }
            bits &= ~((1u << (kWin - n)) - 1u);
        }
        // evaluate the marked samples in order, a round per sample of a lane
        Geo ga, gb;
        float4 a0, a1, b0, b1;
        int ka = 0, kb = 0;
        bool ha = bits != 0, hb;
        if (ha) {                      // the window's lowest marked sample
            const int c = __clz(bits);
            ka = ws + c;
            bits ^= 0x80000000u >> c;
            ga = geo(P, r, (float)ka);
            ga.iz -= z_base;
            cell<DT, STACK>(T, t0, ga.iz, ga.gx, ga.gy, a0, a1);
        }
        while (__any_sync(lanes, ha)) {
            hb = bits != 0;
            if (hb) {
                const int c = __clz(bits);
                kb = ws + c;
                bits ^= 0x80000000u >> c;
                gb = geo(P, r, (float)kb);
                gb.iz -= z_base;
                cell<DT, STACK>(T, t0, gb.iz, gb.gx, gb.gy, b0, b1);
            }
            if (ha && acc.add(P, lut, interp_t<DT, false>(T, a0, a1, ga))) {
                stop = ka + 1;                 // the ray stops after this sample
                live = false;
                bits = 0;
                hb = false;
            }
            ha = hb;
            ka = kb;
            ga = gb;
            a0 = b0;
            a1 = b1;
        }
        if (ws + kWin >= k1) live = false;
    }
    return k0 < k1 ? stop - k0 : 0;
}

template <int DT, int MODE, bool STACK, typename PP, typename TT>
__device__ __forceinline__ int march_tex_win(const PP& P, const TT& T,
                                             const float4* __restrict__ lut, const Ray& r,
                                             Acc<MODE>& acc)
{
    return march_win<DT, MODE, STACK, false>(P, T, lut, r, acc, 0, r.K);
}

// The gathers of sample k + 1 are issued before sample k is interpolated, so
// the texture latency overlaps the arithmetic of the current sample.  The
// loop is unrolled twice with two register sets that swap roles, so a
// pending gather result is only copied when the next sample reuses it.
// Returns the number of samples evaluated.
template <int DT, int MODE, bool STACK, bool KEEP_PAIR = false, typename PP, typename TT>
__device__ __forceinline__ int march_tex(const PP& P, const TT& T, const float4* __restrict__ lut,
                                         const Ray& r, Acc<MODE>& acc)
{
    if (r.K <= 0) return 0;
    if constexpr ((DT == kF16Pair || DT == kI8Pair) && !KEEP_PAIR) {
        // pair texels gathered every sample: the gathers of the next two
        // samples in flight while one is interpolated (three register sets
        // in rotation; 1024^3 FP16 pair MIP, 32 views at 1080p: 44.4 -> 43.3
        // ms, int8 pair unchanged); the same samples, in the same order,
        // with the same arithmetic as the loop below
        const cudaTextureObject_t t0 = T.tex;
        const float last = (float)(r.K - 1);
        Geo ga = geo(P, r, 0.0f), gb = geo(P, r, 1.0f), gc;
        fetch_dec<DT>(T, ga);
        fetch_dec<DT>(T, gb);
        float4 a0, a1, b0, b1, c0, c1;
        cell<DT, STACK>(T, t0, ga.iz, ga.gx, ga.gy, a0, a1);
        cell<DT, STACK>(T, t0, gb.iz, gb.gx, gb.gy, b0, b1);
        float k = 0.0f;             // the sample evaluated next
        for (;;) {
            gc = geo(P, r, k + 2.0f);
            fetch_dec<DT>(T, gc);
            cell<DT, STACK>(T, t0, gc.iz, gc.gx, gc.gy, c0, c1);
            if (acc.add(P, lut, interp_t<DT, true>(T, a0, a1, ga)) || k >= last) break;
            k += 1.0f;
            ga = geo(P, r, k + 2.0f);
            fetch_dec<DT>(T, ga);
            cell<DT, STACK>(T, t0, ga.iz, ga.gx, ga.gy, a0, a1);
            if (acc.add(P, lut, interp_t<DT, true>(T, b0, b1, gb)) || k >= last) break;
            k += 1.0f;
            gb = geo(P, r, k + 2.0f);
            fetch_dec<DT>(T, gb);
            cell<DT, STACK>(T, t0, gb.iz, gb.gx, gb.gy, b0, b1);
            if (acc.add(P, lut, interp_t<DT, true>(T, c0, c1, gc)) || k >= last) break;
            k += 1.0f;
        }
        return (int)(k + 1.0f);
    }
    const cudaTextureObject_t t0 = T.tex;
    const float Kf = (float)r.K;
    Geo ga = geo(P, r, 0.0f), gb;
    fetch_dec<DT>(T, ga);
    float4 a0, a1, b0, b1;
    cell<DT, STACK>(T, t0, ga.iz, ga.gx, ga.gy, a0, a1);
    float kf = 1.0f;            // samples evaluated once the current one is
    for (;;) {
        gb = geo(P, r, kf);
        fetch_dec<DT>(T, gb);
        next_cell<DT, STACK, KEEP_PAIR>(T, t0, ga, a0, a1, gb, b0, b1);
        if (acc.add(P, lut, interp_t<DT, true>(T, a0, a1, ga)) || kf >= Kf) break;
        kf += 1.0f;
        ga = geo(P, r, kf);
        fetch_dec<DT>(T, ga);
        next_cell<DT, STACK, KEEP_PAIR>(T, t0, gb, b0, b1, ga, a0, a1);
        if (acc.add(P, lut, interp_t<DT, true>(T, b0, b1, gb)) || kf >= Kf) break;
        kf += 1.0f;
    }
    return (int)kf;
}

// ---- MIP bounds (8-bit upper-bound codes, BoundScale) ----
// A cell's corners carry codes c_i with L + c_i delta >= v_i; each is read
// as the float y_i = 1 + c_i 2^-15 (exact), and the sample's test value is
// the float trilinear value y of the y_i with the sample's fractions.  With
// Y the exact trilinear value of the y_i, the exact one of the decoded
// corners is U = L + Q (Y - 1), Q = delta 2^15, and U is at least the exact
// trilinear value of the voxels.  The float y is within 18 * 2^-24 of Y
// (three levels of lerps of values below 2, each adding at most 3 * 2^-24 of
// the largest), and the sample's float value v within e of the exact
// trilinear value of the voxels (le = L + e rounded up).  So y < (m - le) /
// Q + 1 - 2^-19 implies v < m: such a sample cannot raise the running
// maximum m.  bound_limit evaluates the right-hand side rounded toward -inf
// at each step (inv_q = 1/Q rounded down, and m - le >= 0 whenever the limit
// is 1 or more, which every y is), so it never exceeds the exact value; for
// m = -inf it is -inf, and with le = +inf (skipping off) it is -inf or NaN:
// every sample is then evaluated.
__device__ __forceinline__ float bound_limit(float m, float2 q)
{
    return __fmaf_rd(__fsub_rd(m, q.x), q.y, 1.0f - 0x1p-19f);
}

// {le, inv_q} of the volume's bound scale (read once per ray).
template <typename TT>
__device__ __forceinline__ float2 bound_consts(const TT& T)
{
    return __ldg(reinterpret_cast<const float2*>(&T.bound_scale->le));
}

// The MIP-bound texels of the cell at slice z (cell slices: slice z packs
// the codes of planes z - 1 and z, low byte the lower plane) whose x/y
// corner is texel (x-1, y-1): one gather returns all eight corners.
template <bool STACK, typename TT>
__device__ __forceinline__ uint4 bound_cell(const TT& T, cudaTextureObject_t tb, int z, float x,
                                            float y)
{
    float yt;
    const int l = plane_layer<STACK>(T, z, y, yt);
    return gather_u32(tb, l, x, yt);
}

// The test value y of a cell's bound texels: each code byte moved into the
// mantissa of 1.0f (bits 8-15: 1 + c 2^-15) by one byte permute, the two
// planes of a texel side by side in a register pair, then interp's
// trilinear interpolation with the lerps of both planes in packed
// instructions (x, then y, then z; the same roundings as interp).  Measured
// against the scalar interpolation: 46.3 -> 45.8 ms for the 32-view MIP
// launch of the 1024^3 cube.
__device__ __forceinline__ float bound_interp(const uint4& b, const Geo& g)
{
    auto planes = [](unsigned w) {
        return pack2(__uint_as_float(__byte_perm(w, 0x3f800000u, 0x7604)),
                     __uint_as_float(__byte_perm(w, 0x3f800000u, 0x7614)));
    };
    const unsigned long long fx = pack2(g.fx, g.fx), fy = pack2(g.fy, g.fy);
    const unsigned long long y0 = lerp2(planes(b.w), planes(b.z), fx);   // row y0, both planes
    const unsigned long long y1 = lerp2(planes(b.x), planes(b.y), fx);   // row y1
    const float2 z = unpack2(lerp2(y0, y1, fy));
    return lerpf(z.x, z.y, g.fz);
}

// MIP over FP32 texture storage with MIP bounds attached: the march of
// march_tex runs over the bound texels (8-bit codes, both planes of a cell
// in one 16-bit texel, one gather a sample), and a sample is evaluated from
// the FP32 texture only when its test value is not below the limit of the
// running maximum (bound_limit), i.e. when it could raise the maximum.  Every
// sample that can change the maximum is evaluated with march_tex's
// arithmetic, so the result and the sample count are march_tex's bit for
// bit.  The gathers of the next two samples are in flight while a sample is
// tested (three register sets in rotation); a pending sample keeps only its
// fractions and gather result, and a candidate's gather coordinates are
// computed again from its index (geo is deterministic), which keeps the
// march at 48 registers (1024^3, 32 views at 1080p: 45.8 -> 44.1 ms against
// one gather ahead; three ahead 46.1 ms).  (Gathering every sample, even in
// the same cell, measured faster than testing for a change of cell and
// keeping the held texels: the test and the selects cost more issue slots
// than the gather.)
struct BoundSample {
    float fx, fy, fz;   // the sample's fractions (geo)
    uint4 u;            // its cell's bound texels
};

template <bool STACK, typename PP, typename TT>
__device__ __forceinline__ int march_tex_bound(const PP& P, const TT& T, const Ray& r,
                                               Acc<VR_MIP>& acc)
{
    if (r.K <= 0) return 0;
    const cudaTextureObject_t tb = T.bound, tf = T.tex;
    const float last = (float)(r.K - 1);     // the last sample's index
    const float2 q = bound_consts(T);
    float lim = bound_limit(acc.m, q);
    // gather the bounds of sample kf (positions past the ray's end stay
    // within a few voxels of the box: the texture clamps their coordinates)
    auto issue = [&](float kf, BoundSample& b) {
        const Geo g = geo(P, r, kf);
        b.fx = g.fx;
        b.fy = g.fy;
        b.fz = g.fz;
        b.u = bound_cell<STACK>(T, tb, g.iz, g.gx, g.gy);
    };
    auto take = [&](const BoundSample& b, float kf) {
        Geo h;
        h.fx = b.fx;
        h.fy = b.fy;
        h.fz = b.fz;
        if (!(bound_interp(b.u, h) < lim)) {
            const Geo g = geo(P, r, kf);
            float4 e0, e1;
            cell<VR_F32, STACK>(T, tf, g.iz, g.gx, g.gy, e0, e1);
            acc.m = fmaxf(acc.m, interp(e0, e1, g));
            lim = bound_limit(acc.m, q);
        }
    };
    BoundSample sa, sb, sc;
    issue(0.0f, sa);
    issue(1.0f, sb);
    float k = 0.0f;             // the sample taken next
    for (;;) {
        issue(k + 2.0f, sc);
        take(sa, k);
        if (k >= last) break;
        k += 1.0f;
        issue(k + 2.0f, sa);
        take(sb, k);
        if (k >= last) break;
        k += 1.0f;
        issue(k + 2.0f, sb);
        take(sc, k);
        if (k >= last) break;
        k += 1.0f;
    }
    return (int)(k + 1.0f);
}

// ---- rendering a cube part by part ----
// A part holds planes [base, base + n) of a larger cube (its slices are the
// part's own: local slice = global slice - base).  Rendering a part marches,
// of each ray of the whole cube, the samples whose cell (floor of the sample
// height) lies in [lo, hi): cells whose two planes are both in the part (the
// first part also takes the cells below plane 0, the last those above the
// top plane, positions a rounding error outside the box).  Sample heights
// are monotone in k, so those samples are one range of k, found by bisection
// with the march's own position arithmetic.

// Cell (floor of the height) of sample k.
template <typename PP>
__device__ __forceinline__ float sample_cell(const PP& P, const Ray& r, int k)
{
    return floorf(fmaf(fmaf((float)k, P.step, r.te), r.dz, r.oz));
}

// First k in [0, K] whose cell satisfies `past` (false before it, true from
// it on: the predicate is monotone in k).
template <typename PP, typename F>
__device__ __forceinline__ int first_k(const PP& P, const Ray& r, F past)
{
    int a = 0, b = r.K;
    while (a < b) {
        const int m = (a + b) >> 1;
        if (past(sample_cell(P, r, m)))
            b = m;
        else
            a = m + 1;
    }
    return a;
}

// Whether any sample of the ray can lie in the part's cells: sample cells
// are monotone in k, so those of the first and last samples bound them all.
template <typename PP>
__device__ __forceinline__ bool may_cross_part(const PP& P, const Ray& r)
{
    const float lo = (float)P.part_lo, hi = (float)P.part_hi;
    const float c0 = sample_cell(P, r, 0), c1 = sample_cell(P, r, r.K - 1);
    const float cmin = fminf(c0, c1), cmax = fmaxf(c0, c1);
    return cmax >= lo && cmin < hi;
}

// Samples [k0, k1) of the part's cells, for a ray going up (dz >= 0) or down.
template <typename PP>
__device__ __forceinline__ void part_range(const PP& P, const Ray& r, int& k0, int& k1)
{
    const float lo = (float)P.part_lo, hi = (float)P.part_hi;
    if (r.dz >= 0.0f) {
        k0 = first_k(P, r, [&](float c) { return c >= lo; });
        k1 = first_k(P, r, [&](float c) { return c >= hi; });
    } else {
        k0 = first_k(P, r, [&](float c) { return c < hi; });
        k1 = first_k(P, r, [&](float c) { return c < lo; });
    }
}

// march_tex over samples [k0, k1) of a part, continuing `acc`; slices are
// shifted to the part's own.  Returns the number of samples evaluated.
template <int DT, int MODE, bool STACK, typename PP, typename TT>
__device__ __forceinline__ int march_part(const PP& P, const TT& T,
                                          const float4* __restrict__ lut, const Ray& r,
                                          Acc<MODE>& acc, int k0, int k1)
{
    if (k0 >= k1) return 0;
    const cudaTextureObject_t t0 = T.tex;
    int k = k0;
    float kf = (float)k0;
    Geo ga = geo(P, r, kf), gb;
    ga.iz -= P.slice_base;
    fetch_dec<DT>(T, ga);
    float4 a0, a1, b0, b1;
    cell<DT, STACK>(T, t0, ga.iz, ga.gx, ga.gy, a0, a1);
    kf += 1.0f;
    for (;;) {
        gb = geo(P, r, kf);
        gb.iz -= P.slice_base;
        fetch_dec<DT>(T, gb);
        next_cell<DT, STACK, false>(T, t0, ga, a0, a1, gb, b0, b1);
        ++k;
        if (acc.add(P, lut, interp_t<DT, true>(T, a0, a1, ga)) || k >= k1) break;
        kf += 1.0f;
        ga = geo(P, r, kf);
        ga.iz -= P.slice_base;
        fetch_dec<DT>(T, ga);
        next_cell<DT, STACK, false>(T, t0, gb, b0, b1, ga, a0, a1);
        ++k;
        if (acc.add(P, lut, interp_t<DT, true>(T, b0, b1, gb)) || k >= k1) break;
        kf += 1.0f;
    }
    return k - k0;
}

// march_tex_bound over samples [k0, k1) of a part (MIP over FP32 texture
// storage with MIP bounds), continuing `acc`; slices shifted to the part's
// own.  The result is march_part's bit for bit (see march_tex_bound).
template <bool STACK, typename PP, typename TT>
__device__ __forceinline__ int march_part_bound(const PP& P, const TT& T, const Ray& r,
                                                Acc<VR_MIP>& acc, int k0, int k1)
{
    if (k0 >= k1) return 0;
    const cudaTextureObject_t tb = T.bound, tf = T.tex;
    const float2 q = bound_consts(T);
    float lim = bound_limit(acc.m, q);
    auto take = [&](const Geo& g, const uint4& u) {
        if (!(bound_interp(u, g) < lim)) {
            float4 e0, e1;
            cell<VR_F32, STACK>(T, tf, g.iz, g.gx, g.gy, e0, e1);
            acc.m = fmaxf(acc.m, interp(e0, e1, g));
            lim = bound_limit(acc.m, q);
        }
    };
    int k = k0;
    float kf = (float)k0;
    Geo ga = geo(P, r, kf), gb;
    ga.iz -= P.slice_base;
    uint4 a = bound_cell<STACK>(T, tb, ga.iz, ga.gx, ga.gy), b;
    kf += 1.0f;
    for (;;) {
        gb = geo(P, r, kf);
        gb.iz -= P.slice_base;
        b = bound_cell<STACK>(T, tb, gb.iz, gb.gx, gb.gy);
        take(ga, a);
        if (++k >= k1) break;
        kf += 1.0f;
        ga = geo(P, r, kf);
        ga.iz -= P.slice_base;
        a = bound_cell<STACK>(T, tb, ga.iz, ga.gx, ga.gy);
        take(gb, b);
        if (++k >= k1) break;
        kf += 1.0f;
    }
    return k - k0;
}

template <int DT>
__device__ __forceinline__ float load_voxel(const void* b, size_t i)
{
    if (DT == VR_F32) return __ldg(static_cast<const float*>(b) + i);
    if (DT == VR_F16) return __half2float(__ldg(static_cast<const __half*>(b) + i));
    return (float)__ldg(static_cast<const signed char*>(b) + i);
}

// Trilinear sample from the bricks at a point already clamped to the box.
// PP supplies bricks, g, scale and offset.
template <int DT, typename PP>
__device__ __forceinline__ float sample_bricks(const PP& P, float px, float py, float pz)
{
    const VolumeGeom& g = P.g;
    const int ix = min((int)px, g.nx - 2);
    const int iy = min((int)py, g.ny - 2);
    const int iz = min((int)pz, g.nz - 2);
    const float fx = px - (float)ix, fy = py - (float)iy, fz = pz - (float)iz;
    const size_t brick = ((size_t)(iz >> kBrickShift) * g.nby + (iy >> kBrickShift)) * g.nbx +
                         (ix >> kBrickShift);
    const size_t base = brick * kBrickVoxels + ((iz & 31) << 10) + ((iy & 31) << 5) + (ix & 31);
    const size_t sx = ((ix & 31) == 31) ? (size_t)(kBrickVoxels - 31) : 1;
    const size_t sy = ((iy & 31) == 31) ? (size_t)g.nbx * kBrickVoxels - 31 * 32 : 32;
    const size_t sz = ((iz & 31) == 31) ? (size_t)g.nbx * g.nby * kBrickVoxels - 31 * 1024 : 1024;
    if (!debug_ok(base + sx + sy + sz < (size_t)g.nbx * g.nby * g.nbz * kBrickVoxels, 2))
        return 0.0f;
    float c000 = load_voxel<DT>(P.bricks, base);
    float c100 = load_voxel<DT>(P.bricks, base + sx);
    float c010 = load_voxel<DT>(P.bricks, base + sy);
    float c110 = load_voxel<DT>(P.bricks, base + sx + sy);
    float c001 = load_voxel<DT>(P.bricks, base + sz);
    float c101 = load_voxel<DT>(P.bricks, base + sz + sx);
    float c011 = load_voxel<DT>(P.bricks, base + sz + sy);
    float c111 = load_voxel<DT>(P.bricks, base + sz + sx + sy);
    if (DT == VR_I8) {
        const float s0 = __ldg(P.scale + iz), o0 = __ldg(P.offset + iz);
        const float s1 = __ldg(P.scale + iz + 1), o1 = __ldg(P.offset + iz + 1);
        c000 = fmaf(c000, s0, o0); c100 = fmaf(c100, s0, o0);
        c010 = fmaf(c010, s0, o0); c110 = fmaf(c110, s0, o0);
        c001 = fmaf(c001, s1, o1); c101 = fmaf(c101, s1, o1);
        c011 = fmaf(c011, s1, o1); c111 = fmaf(c111, s1, o1);
    }
    const float y0z0 = lerpf(c000, c100, fx), y1z0 = lerpf(c010, c110, fx);
    const float y0z1 = lerpf(c001, c101, fx), y1z1 = lerpf(c011, c111, fx);
    return lerpf(lerpf(y0z0, y1z0, fy), lerpf(y0z1, y1z1, fy), fz);
}

// The march with brick gathers; returns the number of samples evaluated.
template <int DT, int MODE, typename PP>
__device__ __forceinline__ int march_bricks(const PP& P, const float4* __restrict__ lut,
                                            const Ray& r, Acc<MODE>& acc)
{
    int k = 0;
    float kf = 0.0f;
    for (; k < r.K; ++k, kf += 1.0f) {
        const float t = fmaf(kf, P.step, r.te);
        const float qx = fminf(fmaxf(fmaf(t, r.dx, r.ox), 0.0f), P.hix);
        const float qy = fminf(fmaxf(fmaf(t, r.dy, r.oy), 0.0f), P.hiy);
        const float qz = fminf(fmaxf(fmaf(t, r.dz, r.oz), 0.0f), P.hiz);
        if (acc.add(P, lut, sample_bricks<DT>(P, qx, qy, qz))) {
            ++k;
            break;
        }
    }
    return k;
}

}  // namespace ray
}  // namespace vr
