"""Device memory through a caller's allocator (bdu_set_allocator; here
PyTorch's caching allocator through Python callbacks), and an injected
allocation failure: the update that needs new memory answers BDU_ENOMEM
before any device work, and the handle stays usable, bit-identical to the
oracle afterwards (FP64)."""
import numpy as np
import pytest
import torch

import oracle as O
from paper_2509_02840_gb300 import bdu, inputs as I

pytestmark = pytest.mark.gpu


def test_injected_allocation_failure_keeps_the_handle_usable():
    state = {"fail": False, "live": 0}

    def alloc(nbytes, dev):
        if state["fail"]:
            return 0
        state["live"] += 1
        return int(torch.cuda.caching_allocator_alloc(nbytes, device=dev))

    def free(ptr, dev):
        state["live"] -= 1
        torch.cuda.caching_allocator_delete(ptr)

    bdu.set_allocator(alloc, free)
    try:
        m, n = 120, 80
        Q, d, e, P = I.factorization(m, n, config=0, which=91)
        with bdu.Factorization(Q, d, e, P, precision=bdu.FP64) as F:
            assert state["live"] > 0
            B, C = I.dense_update(m, n, 0, config=0, r=1)
            F.update(B, C)
            Q, d, e, P, _ = O.update(Q, d, e, P, B, C)
            state["fail"] = True
            B8, C8 = I.dense_update(m, n, 1, config=0, r=8)
            with pytest.raises(bdu.BduError) as err:
                F.update(B8, C8)  # a rank-8 workspace is new memory
            assert err.value.code == 2  # BDU_ENOMEM
            state["fail"] = False
            B, C = I.dense_update(m, n, 2, config=0, r=1)
            F.update(B, C)
            Q, d, e, P, _ = O.update(Q, d, e, P, B, C)
            for a, b in zip(F.read(), (Q, d, e, P)):
                assert np.array_equal(a, b)
        assert state["live"] == 0  # every block went back through the caller's free
    finally:
        bdu.set_allocator(None)
