"""GB300 (sm_103a) hot path of the cascaded lattice Boltzmann method of Liu & He
for 2D microchannel gas flow (arXiv:1603.01955).

The D2Q9 stream-and-collide sweep, its boundaries and the observable reductions
are hand-written CUDA kernels behind the C ABI of ``include/clb.h``; this
package is their thin Python binding (``clb``) and build step (``build``).
"""
from .clb import (  # noqa: F401
    CLB_BF16_SCALED,
    CLB_DRIVE_BODY_FORCE,
    CLB_DRIVE_PRESSURE,
    CLB_FP16_SCALED,
    CLB_FP32_SHIFTED,
    CLB_FP64,
    LIB_PATH,
    Batch,
    Channel,
    CLBError,
    FlowGradient,
    clb_create,
    clb_destroy,
    clb_get_state,
    clb_info,
    clb_observables,
    clb_opts_default,
    clb_set_state,
    clb_step,
    clb_sync,
    flow_rate,
)
