"""B300-native space-charge tracking step (arXiv:2208.02382, ImpactX v22.08).

The compute path is libbeamtrack.so (hand-written sm_103a CUDA kernels behind
the C ABI of include/beamtrack.h); `api` is its thin Python binding.
"""
from .api import (Batch, Beam, Element, Grid, Species, Tracker, lattice_struct,  # noqa: F401
                  twiss_beam, twiss_grad, autotune_batch, distribution_beam, shard_range,
                  objectives, family_grad,
                  torch_allreduce)
from .autograd import TrackObjectives, track_objectives  # noqa: F401
