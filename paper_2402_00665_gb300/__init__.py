"""GB300-native linear BVH with skip connections (arXiv 2402.00665).

The build (Morton codes, radix sort, the modified Apetrei bottom-up pass with
Karras ordering, boxes and skips) and the stackless range query run in
hand-written CUDA kernels for sm_103a, behind the C ABI declared in
``include/lbvh.h``. ``paper_2402_00665_gb300.lbvh`` is the thin Python binding
over that library; ``paper_2402_00665_gb300.inputs`` draws the seeded
synthetic workloads. Importing this package loads nothing: the CUDA library is
loaded (and must be present) on first use of the binding.
"""

__all__ = ["inputs", "lbvh"]
__version__ = "0.1.0"
