"""GB300 (sm_103a) PDLP: restarted primal-dual hybrid gradient for linear programming.

The solver is the CUDA library libpdlp.so behind the C ABI of include/pdlp.h; this
package only marshals arguments to it (see ``binding``).
"""
from .binding import (FP32_BULK, FP64, STATUS_NAMES, PdlpError, SolveResult, default_params,  # noqa: F401
                      gather_bench, kkt, kkt_products_noalloc, load_library, normalized_gap, precondition, solve,
                      solve_batch, solve_instance)
