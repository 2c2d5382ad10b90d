"""GB300-native three-phase MRT colour-gradient lattice Boltzmann step with the
characteristic-line wetting condition (arXiv:2102.04709).

``paper_2102_04709_gb300.lbm3`` is the binding of the C-ABI library (CUDA, sm_103a);
``paper_2102_04709_gb300.workloads`` generates the seeded synthetic inputs.
"""
__all__ = ["lbm3", "workloads"]
