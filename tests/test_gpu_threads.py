"""Contexts on concurrent host threads: two contexts (MIXED sphere at 32^3,
FP64 ellipsoid at 32^3) solve three times each on their own thread and CUDA
stream at the same time.  Every concurrent solve must equal the same
context's sequential solve bit for bit (the kernels reduce in a fixed order)
with the same iteration counts and kernel-launch count (launches are counted
per calling thread)."""
import threading

import numpy as np
import pytest

import kfbim_inputs as ki

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from paper_2303_04992_gb300 import FP64, MIXED, Solver, build  # noqa: E402

build()


def boundary_data(s, seed):
    xyz, comp, _, prim = s.points()
    rows = np.arange(len(comp))
    g = ki.harmonic_curl_field(seed, degree=3)(xyz)[rows, comp - 1][prim]
    return torch.from_numpy(np.ascontiguousarray(g)).cuda()


def run(s, g):
    N3 = s.N ** 3
    phi = torch.zeros(s.n_primary, dtype=torch.float64, device="cuda")
    u = torch.zeros(3 * N3, dtype=torch.float64, device="cuda")
    p = torch.zeros(N3, dtype=torch.float64, device="cuda")
    s.solve(g, phi, None, None, u, p)
    torch.cuda.current_stream().synchronize()
    return phi.cpu().numpy(), u.cpu().numpy(), p.cpu().numpy(), dict(s.last_stats)


def test_two_contexts_on_two_threads():
    solvers = [Solver(ki.sphere(), ki.grid(32), precision=MIXED),
               Solver(ki.ellipsoid(), ki.grid(32), precision=FP64)]
    data = [boundary_data(s, 40 + k) for k, s in enumerate(solvers)]
    ref = [run(s, g) for s, g in zip(solvers, data)]
    assert all(r[3]["gmres_residual"] < 1e-10 and r[3]["kernel_launches"] > 0 for r in ref)

    results = [None, None]
    errors = []
    start = threading.Barrier(2)

    def work(k):
        try:
            stream = torch.cuda.Stream()
            with torch.cuda.stream(stream):
                start.wait(timeout=60)
                results[k] = [run(solvers[k], data[k]) for _ in range(3)]
        except Exception as e:  # reported on the main thread
            errors.append(e)

    threads = [threading.Thread(target=work, args=(k,)) for k in range(2)]
    for t in threads:
        t.start()
    for t in threads:
        t.join(timeout=600)
    assert not any(t.is_alive() for t in threads)
    assert not errors, errors
    for k in range(2):
        for phi, u, p, st in results[k]:
            assert np.array_equal(phi, ref[k][0]), k
            assert np.array_equal(u, ref[k][1]), k
            assert np.array_equal(p, ref[k][2]), k
            assert st == ref[k][3], (k, st, ref[k][3])
