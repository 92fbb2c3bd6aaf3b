"""Seeded synthetic inputs shaped like the workloads of arXiv:1907.01995.

This package is the only code shared by the FP64 oracle and the CUDA path.
It draws data (designs, labels, noise, regularisation weights) and holds none
of RAC-MBADMM's arithmetic: no permutation, no block step, no prox, no KKT.
"""
from .workloads import (  # noqa: F401
    Instance,
    regression_instance,
    lasso_instance,
    elastic_net_instance,
    svm_instance,
    svm_batch,
    warmstart_instance,
    warmstart_family,
    path_instance,
    small_instance,
    sparse_en_instance,
    rbf_svm_data,
)
