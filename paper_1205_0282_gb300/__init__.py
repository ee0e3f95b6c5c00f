"""GB300 bricked volume ray caster (after Hassan, Fluke & Barnes, arXiv:1205.0282).

The rendering path lives in ``libvr.so`` (CUDA, sm_103a) behind the C ABI of
``include/vr.h``; ``paper_1205_0282_gb300.vr`` is its Python binding.  The
binding's names are loaded on first use, so ``paper_1205_0282_gb300.build`` can
be imported (to compile the library) before the library exists.
"""
_EXPORTED = ("VolumeRenderer", "VRError", "VR_OPT_MODE", "VR_OPT_RECT_CULL", "VR_OPT_SKIP_EMPTY",
             "VR_OPT_KERNEL", "VR_KERNEL_TMA", "VR_KERNEL_DIRECT", "VR_KERNEL_TEX", "VR_KERNEL_AUTO",
             "VR_OPT_PRECISION", "VR_PRECISION_F32", "VR_PRECISION_F16", "VR_PRECISION_F8", "vr_render_noalloc",
             "vr_brick", "vr_create", "vr_destroy", "vr_get_brick_minmax", "vr_get_stats",
             "vr_last_error", "vr_load_cube", "vr_plan_brick_rects", "vr_render",
             "vr_reset_stats", "vr_set_camera", "vr_set_option", "vr_set_transfer_function",
             "vr_kd_partition", "vr_kd_order", "vr_set_region", "vr_region_rect", "vr_plan_region_rect",
             "vr_render_rect", "vr_composite_subimages", "vr_load_cube_host", "VR_OPT_DEVICE_BUDGET",
             "Server", "vr_server_create", "vr_server_submit", "vr_server_wait", "vr_server_get_stats",
             "vr_server_destroy", "Codec", "vr_load_cube_codec", "VR_OPT_STEP_MODE")

__all__ = list(_EXPORTED)


def __getattr__(name):
    if name in _EXPORTED:
        from . import vr
        return getattr(vr, name)
    raise AttributeError(name)
