"""Errors measured by the GPU parity tests, collected for a per-workload report (test infrastructure).

Tests call ``record(case, precision, max_rel=..., total_rel=...)``; when the environment variable
CDP_PARITY_REPORT names a file, ``conftest.py`` writes everything recorded to it (JSON) at the end
of the session: per case and precision, max |m_gpu - m_oracle| / max m_oracle over the compared
cells, the relative total-mass error and the number of cells compared.
"""
RESULTS = {}


def record(case: str, precision: int, **figures) -> None:
    key = "fp64" if precision == 0 else "fp32mixed"
    RESULTS.setdefault(case, {})[key] = {k: (float(v) if isinstance(v, float) else v) for k, v in figures.items()}
