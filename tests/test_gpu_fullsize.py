"""Full-size checks in the benchmark's launch configuration, where the oracle
cannot follow the whole state: properties that hold at any size and sampled
outputs the oracle computes one by one.

* the 30-qubit benchmark circuit (40 layers Haar SU(2) + brickwork CZ) through the
  fused blocks (BF16 split, the benchmark's method) and the tile passes: both
  normalised, the two independent paths agree, and the circuit followed by its
  inverse returns to |0...0>;
* QFT-30 on a random basis state: 4096 sampled amplitudes against the closed form
  of Eq. (multiqubitqft);
* the largest state this GPU holds comfortably, 34 qubits complex64 (128 GiB):
  circuit + inverse through both methods, checked through marginals.

Tolerances: complex64 relative L2 <= 1e-5 per path (depth <= 40), so two paths
differ by <= 2e-5 and a circuit and its inverse leave |<0|psi>|^2 >= 1 - 4e-5.
"""
import numpy as np
import pytest
import torch

import workloads as W
from oracle import statevector as SV

pytestmark = pytest.mark.gpu


def _inverse(ops):
    inv = []
    for name, q, params, m in reversed(ops):
        if name == "MAT1":
            inv.append(("MAT1", q, params, np.asarray(m).conj().T))
        elif name == "CZ":
            inv.append((name, q, params, m))
        else:
            raise ValueError(name)
    return inv


def test_bench_circuit_30_qubits_blocks_and_tiled(qs):
    n = 30
    ops = W.layered_haar_cz(n, 40, seed=2001)
    arr = qs.gates_array(ops)
    inv = qs.gates_array(_inverse(ops))
    out = {}
    for name, method in (("blocks", qs.METHOD_BLOCKS_BF16), ("tiled", qs.METHOD_TILED)):
        st = qs.State(n, qs.QS_C64)
        qs.sv_apply_circuit(st, arr, method)
        _, norm = qs.sv_probs(st, marg_mask=1)
        assert abs(norm - 1.0) < 1e-5, (name, norm)
        amps = torch.empty(1 << n, dtype=torch.complex64, device="cuda")
        qs.sv_copy_out(st, out=amps)
        out[name] = amps
        qs.sv_apply_circuit(st, inv, method)           # back to |0...0>
        back = torch.empty(1 << n, dtype=torch.complex64, device="cuda")
        qs.sv_copy_out(st, out=back)
        p0 = float(back[0].abs() ** 2)
        assert p0 > 1 - 4e-5, (name, p0)
        del back
        st.close()
    rel = float((out["blocks"] - out["tiled"]).norm() / out["tiled"].norm())
    assert rel < 2e-5, rel
    del out
    torch.cuda.empty_cache()


def test_qft_30_sampled_closed_form(qs):
    n = 30
    J = W.random_basis_index(n, 2002)
    st = qs.State(n, qs.QS_C64)
    qs.sv_set_basis(st, J)
    qs.sv_apply_circuit(st, W.qft_circuit(n))
    amps = torch.empty(1 << n, dtype=torch.complex64, device="cuda")
    qs.sv_copy_out(st, out=amps)
    st.close()
    K = np.random.default_rng(2002).integers(0, 1 << n, size=4096)
    got = amps[torch.from_numpy(K).cuda()].cpu().numpy().astype(np.complex128)
    ref = SV.qft_amplitudes(n, J, K)
    assert np.linalg.norm(got - ref) / np.linalg.norm(ref) < 1e-5
    assert np.max(np.abs(got - ref)) < 1e-9            # amplitudes are 2^-15 in magnitude
    del amps
    torch.cuda.empty_cache()


@pytest.mark.parametrize("method", ["tiled", "blocks_bf16"])
def test_max_size_34_qubits_round_trip(qs, method):
    n = 34                                             # 2^34 x 8 B = 128 GiB
    m = {"tiled": qs.METHOD_TILED, "blocks_bf16": qs.METHOD_BLOCKS_BF16}[method]
    ops = W.layered_haar_cz(n, 3, seed=3400)
    st = qs.State(n, qs.QS_C64)
    qs.sv_apply_circuit(st, ops, m)
    p, norm = qs.sv_probs(st, marg_mask=0b11)         # FP64 norm of the whole state
    assert abs(norm - 1.0) < 1e-5, norm
    assert float(p[0]) < 0.5                           # the circuit moved the state
    qs.sv_apply_circuit(st, _inverse(ops), m)
    # |<0...0|psi>|^2 >= 1 - sum of the three marginals' weights off their all-zero outcome
    lost = 0.0
    for mask in (0xFFFF, 0xFFFF << 16, 0b11 << 32):
        p, norm = qs.sv_probs(st, marg_mask=mask)
        assert abs(norm - 1.0) < 1e-5, norm
        lost += 1.0 - float(p[0])
    assert lost < 1e-4, lost
    st.close()
    torch.cuda.empty_cache()
