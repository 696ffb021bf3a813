"""GB300-native SDC / MLSDC / PFASST heat-equation solver (arXiv:1307.7867).

The compute path lives in the CUDA library ``libheat3d.so`` (sources under
``csrc/``); :mod:`paper_1307_7867_gb300.heat3d` is its thin ctypes binding.
Importing the package itself loads nothing, so the input generators in
:mod:`paper_1307_7867_gb300.inputs` can be used without a GPU.
"""
