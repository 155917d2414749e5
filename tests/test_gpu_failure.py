"""Failure path of the bounded device-side waits, exercised without letting a wait run out.

The bulk-copy rings of the double-float and s-step engines wait on mbarriers with an iteration
limit; a wait that gives up sets the handle's device error word, and the solve maps it to
MGH_TIMEOUT at its next restart.  Here the word is set from the host (mgh_debug_inject_timeout),
so no kernel waits in vain: the test checks the mapping, that the handle stays usable, and that
handles whose solver does not poll the word refuse the hook.
"""
import numpy as np
import pytest

import oracle as O
import workloads as W
from gpu_common import make_solver, oracle_solver, rel, torch_cuda

pytestmark = pytest.mark.gpu


def _w(precision="mixed32", **kw):
    return W.Workload("fail", 40, 33, 6, 8.0, 2, -30.0, 30.0, "ellipses", 11, levels=3, nu1=1, nu2=1,
                      precision=precision, restart=8, tol=1e-10, **kw)


@pytest.mark.parametrize("arnoldi", ["sstep", "df"])
def test_error_word_gives_timeout_and_the_handle_stays_usable(arnoldi):
    torch = torch_cuda()
    from paper_2107_03679_gb300 import capi
    w = _w()
    p, f, o = oracle_solver(w)
    s = make_solver(w, B=2, maxit=4000, arnoldi=arnoldi)
    s.set_contrast(torch.from_numpy(f).cuda())
    th = W.angles(w)
    b = np.stack([O.rhs(p, f, t) for t in th])
    bt = torch.from_numpy(b).cuda()
    x = torch.zeros_like(bt)
    capi.mgh_debug_inject_timeout(s._h)
    st = capi._lib.mgh_solve(s._h, capi._ptr(bt), 2, capi._ptr(x), None)
    assert st == capi.MGH_TIMEOUT, capi.mgh_status_string(st)
    # the hook is one-shot: the next solve on the same handle converges to the direct solution
    x, infos = s.solve(bt)
    assert all(i["converged"] for i in infos), infos
    for q in range(2):
        assert rel(x.cpu().numpy()[q], O.direct_solve(p, o.D, b[q])) < 1e-5
    s.close()


def test_hook_refused_where_no_solver_polls_the_error_word():
    torch_cuda()
    from paper_2107_03679_gb300 import capi
    for kw in (dict(precision="fp64"), dict(krylov="bicgstab"), dict(arnoldi="fp64")):
        w = _w(precision=kw.pop("precision", "mixed32"))
        s = make_solver(w, B=1, **kw)
        with pytest.raises(capi.MGHError) as e:
            capi.mgh_debug_inject_timeout(s._h)
        assert e.value.status == capi.MGH_NOT_SUPPORTED
        s.close()
