"""GB300-native variational inference for the Bayesian non-negative factorial
HMM (Mysore & Sahani, ICML 2012).

The compute path is the C-ABI library ``libnfhmm.so`` (CUDA, sm_103a) built
from ``csrc/``; :mod:`paper_1206_6468_gb300.nfhmm` is its ctypes binding.
Importing this package does not load the library; importing the binding
does, and raises if the library is missing.
"""

__all__ = ["synth"]
