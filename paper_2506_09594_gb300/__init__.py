"""GB300-native per-iteration low-rank proximal step for high-order tensor
recovery (GNRHTC / GNHTC ADMM of arXiv 2506.09594).

The compute path is the CUDA C-ABI library ``libtr.so`` built from
``csrc/`` (see ``include/tr.h``); ``tr`` is its thin ctypes binding.
``synth`` builds seeded synthetic inputs.
"""
