"""qs_probs_noalloc (probabilities without any device allocation) agrees with sv_probs.

This entry point is for callers that may not allocate device memory; its
reduction scratch is a fixed array in device global memory shared by all
calls.  The test calls it twice in a row through the C ABI on the amplitudes of
an existing state and compares with the allocating entry point (sv_probs)
within the tolerances of the other probability tests: 2e-6 absolute for
complex64 probabilities, 1e-13 for complex128, norms to 1e-12.  This file is
collected last on purpose.
"""
import numpy as np
import pytest
import torch

import workloads as W

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("prec", [0, 1])
@pytest.mark.parametrize("n", [5, 14])
def test_noalloc_matches_sv_probs_twice(qs, n, prec):
    st = qs.State(n, prec)
    qs.sv_apply_circuit(st, W.random_gate_mix(n, 80, seed=900 + n))
    ref, ref_norm = qs.sv_probs(st, fp64=True)
    tol = 1e-13 if prec else 2e-6
    for _ in range(2):   # two calls in a row share (and reuse) the scratch array
        for fp64 in (False, True):
            out = torch.full((1 << n,), -1.0, dtype=torch.float64 if fp64 else torch.float32,
                             device="cuda")
            out, norm = qs.qs_probs_noalloc(st.device_ptr(), n, prec, out=out, fp64=fp64)
            np.testing.assert_allclose(out.double().cpu().numpy(), ref.cpu().numpy(), atol=tol)
            assert abs(norm - ref_norm) < 1e-12
        for mask in (0b11, (1 << n) - 2):
            mref, _ = qs.sv_probs(st, fp64=True, marg_mask=mask)
            k = bin(mask).count("1")
            if k > 12:
                continue
            out = torch.empty(1 << k, dtype=torch.float64, device="cuda")
            out, _ = qs.qs_probs_noalloc(st.device_ptr(), n, prec, out=out, fp64=True, marg_mask=mask)
            np.testing.assert_allclose(out.cpu().numpy(), mref.cpu().numpy(), atol=tol * 4)
    st.close()


def test_noalloc_rejects_sizes_beyond_its_limit(qs):
    n = 14
    st = qs.State(n, 0)
    out = torch.empty(1 << 13, dtype=torch.float64, device="cuda")
    with pytest.raises(qs.QsimError) as e:
        qs.qs_probs_noalloc(st.device_ptr(), n, 0, out=out, fp64=True, marg_mask=(1 << 13) - 1)
    assert e.value.status == qs.QS_EINVAL and "limit" in str(e.value)
    with pytest.raises(qs.QsimError):
        qs.qs_probs_noalloc(st.device_ptr(), 37, 0, out=out)
    st.close()


@pytest.mark.parametrize("prec", [0, 1])
def test_noalloc_largest_marginal_and_optional_outputs(qs, prec):
    # a 12-qubit marginal fills the whole shared histogram and scratch region;
    # out=None computes only the norm; want_norm=False leaves the call asynchronous
    n = 14
    st = qs.State(n, prec)
    qs.sv_apply_circuit(st, W.random_gate_mix(n, 80, seed=950 + prec))
    tol = 1e-13 if prec else 2e-6
    mask = 0b10111111111101          # 12 of the 14 bits
    mref, ref_norm = qs.sv_probs(st, fp64=True, marg_mask=mask)
    for _ in range(2):
        out = torch.full((1 << 12,), -1.0, dtype=torch.float64, device="cuda")
        out, norm = qs.qs_probs_noalloc(st.device_ptr(), n, prec, out=out, fp64=True, marg_mask=mask)
        np.testing.assert_allclose(out.cpu().numpy(), mref.cpu().numpy(), atol=tol * 4)
        assert abs(norm - ref_norm) < 1e-12
        _, norm_only = qs.qs_probs_noalloc(st.device_ptr(), n, prec, out=None)
        assert abs(norm_only - ref_norm) < 1e-12
        p = torch.full((1 << n,), -1.0, dtype=torch.float32, device="cuda")
        _, none = qs.qs_probs_noalloc(st.device_ptr(), n, prec, out=p, want_norm=False)
        assert none is None
        torch.cuda.current_stream().synchronize()
        full, _ = qs.sv_probs(st, fp64=True)
        np.testing.assert_allclose(p.double().cpu().numpy(), full.cpu().numpy(), atol=2e-6)
    st.close()
