"""GB300 fast multipole method for the 3-D Laplace potential and gradient.

``paper_1108_5815_gb300.fmm`` is the binding of the CUDA library (C ABI in
``include/fmm.h``); ``paper_1108_5815_gb300.inputs`` draws the synthetic
particle sets; ``paper_1108_5815_gb300.build`` compiles the library in-tree.
"""
