"""The paper's Fig. 1 program (1-D Laplace on float64[2, N], T steps) on the
GPU through the C ABI, against the FP64 oracle: bit for bit, both rows, on
the figure's own configuration (N = 2033, T = 500) and on shapes that take
the multi-launch path."""
import numpy as np
import pytest
import torch

import oracle
from paper_1902_10345_gb300 import binding, build

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def lib():
    assert torch.cuda.is_available()
    build.build()
    return binding.lib()


@pytest.mark.parametrize("N,T", [(2033, 500), (1, 5), (2, 5), (3, 7), (10, 0), (64, 1), (257, 33), (20000, 40),
                                 (100001, 9)])
def test_fig1_program_bitwise(N, T):
    a = np.random.default_rng(N + T).random((2, N))
    A = torch.from_numpy(a).cuda()
    binding.check(binding.sdfg_laplace1d(A.data_ptr(), N, T, torch.cuda.current_stream().cuda_stream))
    torch.cuda.synchronize()
    assert np.array_equal(A.cpu().numpy(), oracle.laplace1d(a, T))
