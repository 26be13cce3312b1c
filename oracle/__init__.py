"""CPU FP64 oracle of the HODLR-preconditioned GMRES solver -- test infrastructure only.

Only the tests, the smoke check and the benchmark's CPU-baseline leg import this
package.  It shares no code with the CUDA library."""
from .hodlr_oracle import *  # noqa: F401,F403
