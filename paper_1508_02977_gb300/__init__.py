"""GB300-native solver for the P1 finite-element optical-flow model with an
illumination unknown and adaptive per-element regularisation
(Gilliocq-Hirtz & Belhachmi, arXiv 1508.02977).

The compute path is libof.so (CUDA, sm_103a) behind the C ABI of
include/of.h; `ofsolve` is its ctypes binding and `autograd` the
torch.autograd.Function on top.  `synth` makes seeded synthetic inputs and
`partition` holds the subdomain partition rule of Section 3.1.  Importing the
package does not load the library; importing `ofsolve` does, and fails if it
is missing.
"""
__all__ = ["synth", "partition"]
