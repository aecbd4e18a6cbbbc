"""The tensor-core trailing update (FFS_TRAILING_TC): the once-per-panel update of the
blocked state through exact BF16 slices on tcgen05 — the new rows Y = U - C W0_T,
Bot = S^-1 Y and the old rows Top = W0_T - W0_P Bot, real and complex — must give the
double-float state of the direct update to within double-float rounding.  The
conditionals (FP32 outputs of a BF16x3 residual, whose operand split can move by one
BF16 unit when the state moves by a rounding) then agree with the direct path to 1e-7
and with the oracle within the chosen form's 1e-4; cases cover one and several 128-row
tiles of old rows, several 64-row (real) or 32-row (complex) chunks of the new-row
product (its rings wrap), ragged trailing slabs, L-ensemble chains that end inside
panels, the grouped form, real and complex states, and the full-size lattice."""
import numpy as np
import pytest
import torch

from paper_2109_07358_gb300 import ffs
from paper_2109_07358_gb300 import workloads as w
from tests.parity_util import cdf_error, draw_identity, oracle_runs_parallel, window

pytestmark = pytest.mark.gpu

BASE = ffs.FFS_RES_BF16X3 | ffs.FFS_STATE_DF64
TC = BASE | ffs.FFS_TRAILING_TC
SEED = 31337
CASES = {
    "panels": lambda: w.haar(160, 75, seed=9),            # two panel ends, k0 < 128
    "tiles": lambda: w.haar(1000, 300, seed=12),          # k0 up to 256: two row tiles, ragged slabs
    "lattice": lambda: w.square_lattice(16, 16, 100, seed=3),
    "real_tiles": lambda: w.haar(1000, 300, seed=13, complex_=False),
    "anderson": lambda: w.anderson_chain(2048, 200, 1.0, seed=2),
    # k0 up to 608: ten 64-row chunks per new-row product, so every ring of the tensor-core
    # kernels wraps several times
    "real_long": lambda: w.haar(1500, 640, seed=14, complex_=False),
}


@pytest.fixture(scope="module", autouse=True)
def _built():
    from paper_2109_07358_gb300.build import build

    build()
    assert torch.cuda.is_available()


def sampler(U, flags):
    return ffs.Sampler(torch.from_numpy(np.ascontiguousarray(U)).cuda(), flags)


_R = {}


@pytest.mark.parametrize("case", list(CASES))
def test_against_direct_update_and_oracle(case):
    U = CASES[case]()
    B = 70
    if case not in _R:
        _R[case] = oracle_runs_parallel(U, SEED, 0, B)
    recs = _R[case]
    force = torch.tensor(np.stack([r["x"] for r in recs]), dtype=torch.int32, device="cuda")
    probs = {}
    xs = {}
    for name, flags in (("direct", BASE), ("tc", TC)):
        S = sampler(U, flags)
        out = S.sample(B, SEED, force_x=force, probs=True, logp=True)
        xs[name] = S.sample(B, SEED)["x"].cpu().numpy()
        S.sync()
        S.close()
        probs[name] = out["probs"].cpu().double().numpy()
    ref = np.stack([r["probs"] for r in recs])
    d_tc = float(np.abs(probs["tc"] - probs["direct"]).max())
    e_tc = float(np.abs(probs["tc"] - ref).max())
    meas = cdf_error(probs["tc"], recs)
    eps = window(meas, False)
    frac, bad = draw_identity(xs["tc"], recs, eps=eps)
    same = float(np.mean([np.array_equal(a, b) for a, b in zip(xs["tc"], xs["direct"])]))
    print(f"trailing TC {case}: |P_tc - P_direct| {d_tc:.2e}, |P_tc - P_oracle| {e_tc:.2e}, "
          f"samples equal to the direct path {same:.3f}, measured CDF error {meas:.2e}, eps {eps:.2e}")
    assert d_tc <= 1e-7
    assert e_tc <= 1e-4
    assert not bad
    assert same >= 0.95


def test_lensemble_and_grouped():
    V = w.haar(256, 128, seed=5)
    lam = np.ones(128)
    outs = {}
    for name, flags in (("direct", BASE), ("tc", TC)):
        S = sampler(V, flags)
        outs[name] = S.sample_lensemble(lam, 64, SEED, probs=True)
        S.sync()
        S.close()
    assert torch.equal(outs["tc"]["n"], outs["direct"]["n"])
    d = float((outs["tc"]["probs"].double() - outs["direct"]["probs"].double()).abs().max())
    print(f"trailing TC, L-ensemble: max |dP| against the direct path {d:.2e}")
    assert d <= 1e-7
    U = w.haar(400, 150, seed=8)
    g = {}
    for name, flags in (("direct", BASE), ("tc", TC)):
        S = sampler(U, flags | ffs.FFS_FORM_GROUPED)
        g[name] = S.sample(200, SEED, probs=True)["probs"].double()
        S.sync()
        S.close()
    d = float((g["tc"] - g["direct"]).abs().max())
    print(f"trailing TC, grouped form: max |dP| against the direct path {d:.2e}")
    assert d <= 1e-7


def test_full_size_lattice():
    U = w.lattice_64x64_N1024(0)
    recs = oracle_runs_parallel(U, 0, 0, 4)
    S = sampler(U, TC)
    force = torch.tensor(np.stack([r["x"] for r in recs]), dtype=torch.int32, device="cuda")
    out = S.sample(4, 0, force_x=force, probs=True)
    S.sync()
    S.close()
    P = out["probs"].cpu().double().numpy()
    err = max(float(np.abs(P[b] - recs[b]["probs"]).max()) for b in range(4))
    print(f"trailing TC, 64x64 lattice teacher-forced: max |dP| = {err:.2e}")
    assert err <= 1e-4


def test_unsupported_combinations():
    Uc = torch.from_numpy(w.haar(64, 40, seed=1)).cuda()
    for U, flags in ((Uc, ffs.FFS_RES_BF16X3 | ffs.FFS_STATE_FP64 | ffs.FFS_TRAILING_TC),
                     (Uc, ffs.FFS_RES_FP32 | ffs.FFS_STATE_DF64 | ffs.FFS_TRAILING_TC),
                     (Uc, TC | ffs.FFS_TAIL_UNBLOCKED)):
        with pytest.raises(ffs.FFSError) as e:
            ffs.Sampler(U, flags)
        assert e.value.code == ffs.FFS_E_UNSUPPORTED
