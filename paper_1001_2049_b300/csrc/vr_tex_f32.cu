// vr_tex_f32.cu -- the texture-gather kernels (whole cube and cube part)
// instantiated for one texel format (see vr_tex_kernel.cuh).
#include "vr_tex_kernel.cuh"

namespace vr {

cudaError_t launch_tex_f32(const MarchParams& p, const TexParams& t, int mode, int cfg,
                           cudaStream_t s)
{
    return tex::launch_dt<VR_F32>(p, t, mode, cfg, s);
}

cudaError_t launch_part_f32(const MarchParams& p, const TexParams& t, int mode,
                            cudaStream_t s)
{
    return tex::launch_part_dt<VR_F32>(p, t, mode, s);
}

// the checked build's device word of this translation unit
VR_DEBUG_ACCESSOR(debug_flags_tex_f32)

}  // namespace vr
