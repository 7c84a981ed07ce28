"""Plan kernels (Sec. 4.1.2) bit-exact against the oracle's TILE arrays."""
import numpy as np
import pytest
import torch

import inputs
from tests.gpu_helpers import check_tiles, make_plan
from tests.test_oracle_pins import CASES

pytestmark = pytest.mark.gpu


def _csr_from_row_ptr(row_ptr, n_cols=1000, seed=0):
    row_ptr = np.asarray(row_ptr, np.int64)
    lens = np.diff(row_ptr).tolist()
    return inputs.row_lengths_csr(lens, max(n_cols, max(lens + [1])), seed)


@pytest.mark.parametrize("name,row_ptr", CASES)
@pytest.mark.parametrize("sigma", [14, 7, 4, 1])
def test_plan_special(cuda_device, name, row_ptr, sigma):
    a = _csr_from_row_ptr(row_ptr)
    p, _ = make_plan(a, sigma)
    check_tiles(p, a, sigma)


@pytest.mark.parametrize("seed", range(4))
@pytest.mark.parametrize("sigma", [14, 7, 3])
def test_plan_random(cuda_device, seed, sigma):
    a = inputs.random_sparse(500 + 131 * seed, 300, 0.02 * (seed + 1), seed, empty_frac=0.3)
    p, _ = make_plan(a, sigma)
    check_tiles(p, a, sigma)


@pytest.mark.parametrize("sigma", [14, 7])
def test_plan_rmat14(cuda_device, sigma):
    a = inputs.rmat_transition(14, 16, 1)
    p, _ = make_plan(a, sigma)
    ref = check_tiles(p, a, sigma)
    marked = (ref["tile_y"][:-1] & 0x80000000) != 0
    assert marked.any() and (~marked).any()


def test_plan_stress_variants(cuda_device):
    base = inputs.rmat_uniform(16, 16, 3, 3)
    for a in (base, inputs.empty_rows(base, 0.3, 4), inputs.add_hubs(base, 4, 20000, 60000, 5),
              inputs.erdos_renyi(1 << 16, 16, 6)):
        p, _ = make_plan(a, 14)
        check_tiles(p, a, 14)


def test_plan_non_square(cuda_device):
    a = inputs.random_sparse(700, 2000, 0.01, 3, empty_frac=0.1)
    p, _ = make_plan(a, 14)
    check_tiles(p, a, 14)
    b = inputs.random_sparse(3000, 40, 0.05, 4, empty_frac=0.5)
    p, _ = make_plan(b, 14)
    check_tiles(p, b, 14)


def test_plan_full_rmat22(cuda_device):
    """Configuration 2(a) at full size: R-MAT scale 22, edge factor 16."""
    a = inputs.rmat_uniform(22, 16, 3, 3)
    p, _ = make_plan(a, 14)
    check_tiles(p, a, 14)


def test_plan_rejects_bad_row_ptr(cuda_device):
    import paper_2605_07391_gb300 as mb
    row_ptr = torch.tensor([0, 2, 5], dtype=torch.int32, device="cuda")
    col = torch.zeros(4, dtype=torch.int32, device="cuda")
    with pytest.raises(mb.MerbitError) as e:
        mb.plan(row_ptr, col)     # row_ptr[n] = 5 != nnz = 4
    assert e.value.status == 1
