"""GB300-native energy and forces of an ANI-2x-style neural network potential.

The computation is the NNP term of NNP/MM (Galvelis et al., Sec. 2, Eqs. 1-3):
neighbour search, the ANI featurizer, per-element atomic networks with an
ensemble mean, and forces by a hand-written reverse pass, all in CUDA kernels
for sm_103a behind the C ABI of include/nnp.h.

* ``paper_2201_08110_gb300.nnp``: the Python binding (NNP handle, autograd).
* ``paper_2201_08110_gb300.build``: builds libnnp.so in-tree.
* ``paper_2201_08110_gb300.workloads``: seeded synthetic inputs.

Importing this package loads nothing; ``nnp.load_library()`` (called by the
NNP constructor) raises if the library has not been built.
"""

__all__ = ["nnp", "build", "workloads"]
