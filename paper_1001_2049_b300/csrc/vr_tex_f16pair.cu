// vr_tex_f16pair.cu -- the texture-gather kernels (whole cube and cube part)
// instantiated for one texel format (see vr_tex_kernel.cuh).
#include "vr_tex_kernel.cuh"

namespace vr {

cudaError_t launch_tex_f16pair(const MarchParams& p, const TexParams& t, int mode, int cfg,
                               cudaStream_t s)
{
    return tex::launch_dt<kF16Pair>(p, t, mode, cfg, s);
}

cudaError_t launch_part_f16pair(const MarchParams& p, const TexParams& t, int mode,
                                cudaStream_t s)
{
    return tex::launch_part_dt<kF16Pair>(p, t, mode, s);
}

// the checked build's device word of this translation unit
VR_DEBUG_ACCESSOR(debug_flags_tex_f16pair)

}  // namespace vr
