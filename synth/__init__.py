"""Seeded synthetic inputs shared by the oracle and the CUDA path (inputs only)."""
from .generate import Problem, make_problem, WORKLOADS, df_factors  # noqa: F401
from .casci import ActiveSpace, strings  # noqa: F401
