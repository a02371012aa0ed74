"""GB300 (sm_103a) Hamilton-Jacobi safe-set solver for the method of
arXiv 2101.05916 (decomposed, warm-started, coarse-to-fine HJ reachability).

Importing the package loads nothing: `paper_2101_05916_gb300.hj` binds the CUDA
library (libhj_gb300.so, built by `paper_2101_05916_gb300.build`), and
`paper_2101_05916_gb300.workloads` describes the synthetic inputs.
"""
__all__ = ["hj", "workloads", "build"]
