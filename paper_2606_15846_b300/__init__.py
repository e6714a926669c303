"""FlashNav batched bitmap simulator on B300 (sm_103a).

The CUDA library is loaded lazily by :mod:`paper_2606_15846_b300.flashnav`;
importing the package itself loads nothing, so the input generators in
:mod:`paper_2606_15846_b300.workloads` can be used without a GPU.
"""
