"""The profiling-case runner: its arguments, and a loud failure without a CUDA device (no fallback)."""
import pytest

torch = pytest.importorskip("torch")


def test_needs_a_gpu():
    import profile_cases

    if torch.cuda.is_available():
        pytest.skip("a CUDA device is present")
    with pytest.raises(SystemExit, match="CUDA device"):
        profile_cases.main(["c5", "--problem", "3", "--prec", "fp64", "--reps", "1"])


def test_rejects_unknown_cases():
    import profile_cases

    with pytest.raises(SystemExit):
        profile_cases.main(["c9"])
