"""B300-native ray caster for noisy RA x Dec x frequency spectral cubes.

The render path (paper §3.1, process item 3: every output pixel becomes a
ray, mapped to RGBA through a pre-selected transfer function) runs in the
CUDA kernels of ``libvr.so`` behind the C ABI of ``include/vr.h``; this
package is the thin Python binding (``api``), the nvcc build (``build``),
the seeded synthetic inputs (``synth``) and host-side control: the
continuous-batching server (``serve``) and part-by-part streaming of cubes
larger than the device (``stream``).
"""
from .api import (CAMERA_DTYPE, DTYPES, MODES, Request, Volume, batch_autotune,  # noqa: F401
                  batch_shapes, batch_workspace, get_batch_config, integrate_partials,
                  mip_bounds_bytes, render_batch, render_init, set_batch_config,
                  texture_bytes, volume_bytes)
from ._lib import VRError, load  # noqa: F401
