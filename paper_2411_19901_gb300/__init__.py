"""GB300-native memory-efficient label propagation (arxiv 2411.19901).

The compute path is the CUDA library ``liblpa.so`` (sources in ``csrc/``, C ABI in
``include/lpa.h``); :mod:`.lpa` is its thin ctypes binding, :mod:`.build` compiles it and
:mod:`.tune` times the launch choices that never change a result.
"""
from .lpa import (  # noqa: F401
    LPA_BM, LPA_EXACT, LPA_GRAPH, LPA_MG, LPA_MG_UNCLAMPED, LPA_MODULARITY, LPA_PRUNE,
    LPA_RESCAN,
    LPA_TIMING, LPA_VALIDATE, LpaError, Plan, Server, detect,
    lpa_batch_detect, lpa_detect, lpa_detect_ex, lpa_detect_host, lpa_launch_count, lpa_modularity, lpa_modularity_ex,
    lpa_modularity_workspace_size, lpa_options, lpa_options_init, lpa_plan_create,
    lpa_plan_destroy, lpa_plan_run, lpa_plan_sweep, lpa_release_memory, lpa_stats, lpa_tuning,
    lpa_version, lpa_workspace_size, lpa_workspace_size_ex, make_options, modularity,
)
from . import tune  # noqa: F401,E402
