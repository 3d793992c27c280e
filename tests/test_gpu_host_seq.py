"""GPU tests of ps_solve_host_seq: a sequence of solves from host memory whose copies
overlap the neighbouring problems' solves. Every p is bit-identical to the
device-buffer solve of the same f (same kernels, same order of operations), and each
problem's ps_info is its own; plans outside the chunked pipeline take the
one-after-another path with the same results."""

import numpy as np
import pytest

from oracle import solve as S
from paper_1802_10323_gb300 import synth

pytestmark = pytest.mark.gpu


def _problems(shape, count, seed):
    rng = np.random.default_rng(seed)
    return [rng.uniform(-1, 1, shape) * (1 + s) for s in range(count)]


SEQ = [((6, 128, 128), "fp32_refine", 1e-10, 6, 5),   # chunked pipeline, one correction each
       ((6, 128, 128), "fp32_refine", 1e-13, 8, 3),   # several corrections per problem
       ((8, 128, 256), "fp32_refine", 1e-10, 0, 4),   # loop ends at pass 0
       ((12, 24, 32), "fp64", 1e-10, 6, 3),           # no pipeline: one after another
       ((6, 128, 128), "fp32_refine", 1e-10, 6, 1)]


@pytest.mark.parametrize("shape,precision,rtol,max_iter,count", SEQ,
                         ids=[f"{'x'.join(map(str, s))}-{p}-{r:g}-{m}-x{c}" for s, p, r, m, c in SEQ])
def test_sequence_matches_single_solves(lib, shape, precision, rtol, max_iter, count):
    import torch
    nz, ny, nx = shape
    bcs = ("P", "NN", "DD")
    zf = synth.tanh_faces(nz, 1.0, 1.5)
    plan = lib.Plan(nx, ny, nz, 1.0 / nx, 1.0 / ny, zf=zf, bcs=bcs, precision=precision,
                    rtol=rtol, max_iter=max_iter)
    fs = _problems(shape, count, 5 + count)
    fh = [torch.from_numpy(f.copy()).pin_memory() for f in fs]
    ph = [torch.full(shape, float("nan"), dtype=torch.float64).pin_memory() for _ in fs]
    fd = [torch.empty(shape, dtype=torch.float64, device="cuda") for _ in range(2)]
    pd = [torch.empty(shape, dtype=torch.float64, device="cuda") for _ in range(2)]
    infos = plan.solve_host_seq(fh, ph, fd, pd)
    assert len(infos) == count
    for s, f in enumerate(fs):
        info = lib.info_tensor()
        p_dev = plan.solve(torch.as_tensor(f, device="cuda").contiguous(), info=info)
        torch.cuda.synchronize()
        ref = lib.read_info(info)
        assert (infos[s].status, infos[s].iterations) == (ref.status, ref.iterations), s
        assert infos[s].rel_residual == ref.rel_residual, s
        assert np.array_equal(ph[s].numpy(), p_dev.cpu().numpy()), s
    if max_iter == 0:
        assert all(i.iterations == 0 for i in infos)
    if rtol < 1e-12:
        assert all(i.iterations >= 2 for i in infos)
    # the last problem against the oracle
    q = S.solve(fs[-1], 1.0 / nx, 1.0 / ny, zf, *bcs)
    err = np.abs(ph[-1].numpy() - q).max() / np.abs(q).max()
    assert err <= (1e-12 if precision == "fp64" else (1e-5 if max_iter == 0 else 1e-8)), err
    plan.close()


def test_sequence_into_one_output_keeps_the_last(lib):
    """p_host entries may repeat: the copies out run in order, so one buffer ends with
    the last problem's p; the inputs are copied in from distinct host buffers."""
    import torch
    shape = (6, 128, 128)
    nz, ny, nx = shape
    plan = lib.Plan(nx, ny, nz, 1.0 / nx, 1.0 / ny, zf=synth.tanh_faces(nz, 1.0, 1.5),
                    bcs=("P", "P", "NN"), precision="fp32_refine", rtol=1e-10, max_iter=4)
    fs = _problems(shape, 4, 3)
    fh = [torch.from_numpy(f.copy()).pin_memory() for f in fs]
    out = torch.zeros(shape, dtype=torch.float64).pin_memory()
    fd = [torch.empty(shape, dtype=torch.float64, device="cuda") for _ in range(2)]
    pd = [torch.empty(shape, dtype=torch.float64, device="cuda") for _ in range(2)]
    plan.solve_host_seq(fh, [out] * 4, fd, pd)
    last = plan.solve(torch.as_tensor(fs[-1], device="cuda").contiguous())
    torch.cuda.synchronize()
    assert np.array_equal(out.numpy(), last.cpu().numpy())
    plan.close()


def test_sequence_refuses_overlapping_slots(lib):
    """The four device buffers must be disjoint; count 0 does nothing."""
    import torch
    shape = (6, 128, 128)
    nz, ny, nx = shape
    plan = lib.Plan(nx, ny, nz, 1.0 / nx, 1.0 / ny, zf=synth.tanh_faces(nz, 1.0, 1.5),
                    bcs=("P", "P", "NN"), precision="fp32_refine", rtol=1e-10, max_iter=4)
    fh = [torch.zeros(shape, dtype=torch.float64).pin_memory()]
    ph = [torch.zeros(shape, dtype=torch.float64).pin_memory()]
    a = torch.empty(shape, dtype=torch.float64, device="cuda")
    b = torch.empty_like(a)
    c = torch.empty_like(a)
    with pytest.raises(lib.PoissonError, match="overlap"):
        plan.solve_host_seq(fh, ph, [a, b], [c, a])
    assert plan.solve_host_seq([], [], [a, b], [c, torch.empty_like(a)]) == []
    plan.close()
