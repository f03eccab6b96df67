"""GB300-native population-wide evaluation of NEAT genomes (tensorized NEAT,
Section 3.3: transform once, then forward the whole population).

The compute path is the C-ABI CUDA library ``libneat.so`` (see
``include/neat.h``); ``paper_2404_01817_gb300.neat`` is its thin Python
binding.  ``paper_2404_01817_gb300.workloads`` draws seeded synthetic inputs.
"""
__all__ = ["neat", "workloads"]
