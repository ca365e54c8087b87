"""GB300 ensemble MHD time-stepper (decoupled Elsaesser scheme, Algorithm 1).

The compute path is ``libmhde.so`` (hand-written CUDA for sm_103a behind the C
ABI of ``include/mhde.h``); :mod:`.binding` marshals arguments only.
"""
from .binding import (  # noqa: F401
    Library, load_library, Options, Sizes, Stats, MhdeError, EnsembleSolver, library_path,
    declared_functions, block_gram, block_gram_f32, block_combine_f32, block_gram_noalloc, fp64_fma_rate, advance_many, PREC_FP64, PREC_MIXED,
)


def energy_function():
    """The torch.autograd.Function of the ensemble energy (imports torch)."""
    from .autograd import EnsembleEnergy
    return EnsembleEnergy
