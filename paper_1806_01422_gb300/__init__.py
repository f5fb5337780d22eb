"""GB300-native matrix-free spectral-element operators for viscous Burgers and
their discrete adjoint (arXiv:1806.01422), behind the C ABI of include/sem.h.

    from paper_1806_01422_gb300 import Sem, SemMisfit
"""
from .api import Sem, SemBatch, SemMisfit, ckpt_plan, SCHEMES, PRECISIONS, CKPT  # noqa: F401
