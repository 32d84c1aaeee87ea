"""GB300 (sm_103a) Anti-Reflective deblurring library.

The CUDA binding lives in ``paper_1211_0393_gb300.ar`` and is imported on
demand, so that the seeded input generators in ``workloads`` can be used
without a GPU.
"""
