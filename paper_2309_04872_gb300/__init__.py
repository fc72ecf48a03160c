"""GB300-native lattice Boltzmann warm-plasma wakefield solver
(arXiv 2309.04872): CUDA library liblbpwfa.so and its thin binding."""
from .lbpwfa import (FP16S, FP32, FP64, LEC, OPEN, PERIODIC, WARMC, Batch, LbpwfaError, Run,  # noqa: F401
                     library_path, load_library, make_params)


def witness_field(*args, **kw):
    """See wake_grad.witness_field (imports torch on first use)."""
    from .wake_grad import witness_field as _wf
    return _wf(*args, **kw)
