"""GB300-native (sm_103a) 3D-Gaussian submap registration: the differentiable
splat rasteriser and on-device pose optimisation behind LoopSplat's 3DGS
registration (arXiv 2408.10154, Sec. 3.2), as hand-written CUDA kernels
behind the C ABI of include/gsreg.h.

``gsreg`` is the Python binding (argument marshalling only); ``synth`` draws
seeded synthetic workloads; ``build`` compiles the library in-tree."""
from .gsreg import (Context, Gaussians, GsError, Server, default_options, gs_bin, gs_fuse, gs_loss, gs_pose_step,  # noqa: F401
                    gs_probe_fp32, gs_project, gs_register, gs_register_async, gs_register_batch, gs_register_gradient,
                    gs_register_batch_async, gs_render, gs_render_backward, gs_render_backward_saved,
                    gs_render_noalloc, gs_render_saved, gs_overlap_ratio,
                    gs_sort_u32, gs_track_loss, gs_transform, gs_transform_batch, load, split_views)
