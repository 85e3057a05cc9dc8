"""FP64 CPU oracle of the 6-D spectral transport step.

Test infrastructure only: the tests, the smoke check and the bench's CPU
baseline leg call it; the CUDA library and its binding never do.
"""
from .transport import Grid, Problem, exact_free_streaming  # noqa: F401
