"""The profiling runner (`python -m paper_2111_03541_gb300.cases`) on small
cases: every workload it offers runs through libmf and reports its kernels."""
import pytest

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def cases():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2111_03541_gb300 import cases
    return cases


@pytest.mark.parametrize("argv, expect", [
    (["elastic", "--n", "6", "--prec", "mixed", "--reps", "2"], "mixed_elem"),
    (["elastic", "--n", "6", "--prec", "fp64", "--reps", "2"], "elem_elastic_q1_fp64"),
    (["thermal-grf", "--n", "12", "--reps", "2", "--pcg-iters", "5"], "gather_scalar"),
    (["oseen", "--n", "8", "--reps", "2"], "gather_oseen"),
    (["cnn", "--n", "9", "--reps", "2"], "cnn_conv2"),
])
def test_cases_run(cases, capsys, argv, expect):
    cases.main(argv)
    out = capsys.readouterr().out
    assert expect in out
