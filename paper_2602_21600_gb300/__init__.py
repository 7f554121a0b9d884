"""AQR-HNSW query path on one GB300 GPU (sm_103a).

``paper_2602_21600_gb300.aqr`` binds the C ABI of ``libaqr.so``
(``include/aqr.h``); the CUDA kernels live in ``csrc/``.
"""

from .aqr import AqrError, Context, lib, library_path  # noqa: F401
