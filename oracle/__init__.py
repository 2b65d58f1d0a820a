"""FP64 CPU oracle for the NeuralVDB hot path -- TEST INFRASTRUCTURE ONLY.

Plain, slow, obviously-correct numpy implementation of what the CUDA path
computes: the VDB [Hash,5,4,3] tree build (Section 3.1), the Fourier feature
encoding (Section 3.2.2, Eq. 2), the classifier/regressor MLPs and their
losses (Eq. 1 and Section 3.3.1), their gradients and the Adam update
(Section 3.2), sparse-field training by uniform sampling (Section 3.2.1),
source-embedding patches (Section 3.3.2), the hierarchical top-down decode
(Section 3.5, offline sequential access) and point queries on
[Hash,5,4,NN(3)] (Section 3.5, online random access).

Only the test suite, ``__graft_entry__.smoke()`` and the CPU-baseline leg of
``bench.py`` may import this package.  The product (the C-ABI library and its
Python binding) never does, and shares no code with it: the only common
module is ``fixtures/`` (seeded input generators, none of the method's
arithmetic).

Random numbers the method draws (initial weights, the Fourier matrix B,
training-sample indices) come from two counter-based generators implemented
here from their published definitions (SplitMix64, Philox4x32-10), pinned by
known-answer values in the tests.
"""
from . import rng, vdb, nets, codec, blob  # noqa: F401
