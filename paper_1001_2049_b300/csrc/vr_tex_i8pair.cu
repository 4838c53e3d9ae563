// vr_tex_i8pair.cu -- the texture-gather kernels (whole cube and cube part)
// instantiated for one texel format (see vr_tex_kernel.cuh).
#include "vr_tex_kernel.cuh"

namespace vr {

cudaError_t launch_tex_i8pair(const MarchParams& p, const TexParams& t, int mode, int cfg,
                              cudaStream_t s)
{
    return tex::launch_dt<kI8Pair>(p, t, mode, cfg, s);
}

cudaError_t launch_part_i8pair(const MarchParams& p, const TexParams& t, int mode,
                               cudaStream_t s)
{
    return tex::launch_part_dt<kI8Pair>(p, t, mode, s);
}

// the checked build's device word of this translation unit
VR_DEBUG_ACCESSOR(debug_flags_tex_i8pair)

}  // namespace vr
