"""GB300-native hot path of the coupled PINN-LBM droplet method (arXiv 2504.10539).

The compute lives in the CUDA library ``libpinnlbm.so`` behind the C ABI in
``include/pinnlbm.h``; ``paper_2504_10539_gb300.binding`` marshals arguments to
it.  ``workloads`` draws the seeded synthetic inputs.
"""
__all__ = ["workloads", "binding"]
