"""Fused 5-qubit blocks on the tensor cores (tcgen05) vs the FP64 oracle.

Error budget (stated as numbers, relative L2 of the final state):
* TF32 split: each operand keeps ~22 mantissa bits after the hi/lo split
  (2^-22 relative); the tensor cores accumulate in FP32, and that rounding
  grows about linearly with the number of blocks: measured ~6e-7 for 8-13
  blocks and 1.3e-5 for the 151 blocks of a depth-60 20-qubit circuit (per
  block ~8e-8); asserted <= 1e-5 (<= 13 blocks) and <= 2e-5 (151 blocks);
* BF16 split: ~16 mantissa bits per operand (2^-17 ~ 7.6e-6 per block):
  measured ~1.1e-5 for 8-13 blocks and 4.2e-5 for 151 blocks; asserted
  <= 1e-4 and <= 1e-4.
The measured errors are printed (pytest -s) for the record.
"""
import numpy as np
import pytest

import workloads as W
from oracle import statevector as SV

pytestmark = pytest.mark.gpu

TOL = {2: 1e-5, 3: 1e-4}
TOL_DEEP = {2: 2e-5, 3: 1e-4}


def _run(qs, n, ops, method, psi0=None):
    st = qs.State(n, qs.QS_C64)
    if psi0 is not None:
        qs.sv_copy_in(st, psi0.astype(np.complex64))
    stats = qs.sv_apply_circuit(st, ops, method)
    out = qs.sv_copy_out(st)
    st.close()
    return out, stats


@pytest.mark.parametrize("method", [2, 3])
@pytest.mark.parametrize("n", [12, 13, 16])
def test_blocks_random_gate_mix(qs, n, method):
    ops = W.random_gate_mix(n, 120, seed=700 + n)
    psi0 = W.random_state(n, W.rng(n)).astype(np.complex64).astype(np.complex128)
    ref = SV.apply_circuit(psi0.copy(), n, ops)
    out, stats = _run(qs, n, ops, method, psi0)
    err = np.linalg.norm(out - ref) / np.linalg.norm(ref)
    print(f"n={n} method={method} blocks={stats['passes']} rel_l2={err:.2e}")
    assert err <= TOL[method], err


@pytest.mark.parametrize("method", [2, 3])
def test_blocks_depth60_n20(qs, method):
    # the 32-qubit workload's circuit family at 20 qubits (seed 3002), checked in full
    n = 20
    ops = W.layered_haar_cz(n, 60, seed=3002)
    ref = SV.apply_circuit(SV.basis(n), n, ops)
    out, stats = _run(qs, n, ops, method)
    err = np.linalg.norm(out - ref) / np.linalg.norm(ref)
    print(f"depth-60 n=20 method={method} blocks={stats['passes']} rel_l2={err:.2e}")
    assert err <= TOL_DEEP[method], err


def test_blocks_qft_closed_form(qs):
    n = 14
    J = W.random_basis_index(n, 77)
    st = qs.State(n, qs.QS_C64)
    qs.sv_set_basis(st, J)
    qs.sv_apply_circuit(st, W.qft_circuit(n), 2)
    out = qs.sv_copy_out(st)
    st.close()
    ref = SV.qft_amplitudes(n, J)
    assert np.linalg.norm(out - ref) / np.linalg.norm(ref) <= 1e-5


def test_blocks_reject_unsupported(qs):
    st = qs.State(8, qs.QS_C64)
    with pytest.raises(qs.QsimError) as e:
        qs.sv_apply_circuit(st, [("H", (0,), (), None)], 2)
    assert e.value.status == qs.QS_EUNSUPPORTED
    st.close()
