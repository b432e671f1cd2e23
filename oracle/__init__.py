"""Plain FP64 CPU oracle of the inaccessibility measure field (IMF), arXiv 2002.07627.

TEST INFRASTRUCTURE ONLY: imported by `tests/`, by `__graft_entry__.smoke()` and by the
`cpu_baseline` / `--impl reference` legs of `bench.py`. The product path (the CUDA library and
its binding) never imports it, and it imports nothing from the product path except the seeded
input generators, which hold none of the method's arithmetic.

`imf_oracle.c` holds the literal definitions (rotation resampling, direct FP64 collision sums,
brute-force sweep and minimum); `ref.py` orchestrates them in the order of Algorithm 1 and adds
the normalisation, allowance and sensitivity penalty in NumPy FP64; `brute.py` is an
independent set-based brute force for tiny binary grids used to pin the C code.

Parity status: every function is pinned by `tests/test_oracle_*.py` against closed forms,
hand-worked examples, invariants and the independent brute force, except the end-to-end
effect of the penalty on a full topology optimisation run, which needs the paper's FEA and tool
geometry ("parity unpinned" for that use only; the penalty formula itself is pinned).
"""
from .ref import (  # noqa: F401
    quat_to_matrix, rotate_indicator, resample_tool, collision, sweep, erode, imf, imf_subblock, finalize,
    penalize, point_query, rho_obstacle, sharp_sample, process_plan, lib,
)
