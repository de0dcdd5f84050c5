"""Many problems in one CUDA graph (one stream per problem): every problem's
pass from the graph replay equals the same pass run alone, bit for bit (the
same kernels on the same inputs; only their scheduling differs)."""
import pytest
import torch

from synthetic import batch32_problem, flatten_mlp, mlp_params

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def A():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2310_04166_gb300 as mod
    from paper_2310_04166_gb300 import _lib
    _lib.load()
    return mod


def _problems(A, ks, form, n_samples):
    from paper_2310_04166_gb300.batch import Problem
    out = []
    for k in ks:
        p = batch32_problem(k)
        ham = A.Hamiltonian(p["h"], p["g"], p["e_nuc"], p["n_alpha"], p["n_beta"])
        params = torch.tensor(flatten_mlp(mlp_params(p["seed"], p["n"], p["width"], p["n_hidden"])), device="cuda")
        out.append(Problem(ham, A.Model.mlp(p["n"], p["width"], p["n_hidden"], params, form=form), n_samples, 7 + k))
    return out


@pytest.mark.parametrize("form", ["fp32", "bf16"])
def test_graph_of_problems_equals_each_problem_alone(A, form):
    from paper_2310_04166_gb300.batch import BatchedStep
    ks = [1, 5, 7, 14, 16, 12]
    batched = _problems(A, ks, form, 20_000)
    alone = _problems(A, ks, form, 20_000)
    bs = BatchedStep(batched).capture()  # one eager pass (Philox counter 0), then the recording
    bs.replay()                          # the recorded pass with counter 1
    for p in alone:
        p.step()
        p.step()
    torch.cuda.synchronize()
    for a, b in zip(batched, alone):
        k = int(a.nu.item())
        assert k == int(b.nu.item()) and k > 0
        assert torch.equal(a.x[:k], b.x[:k]) and torch.equal(a.cnt[:k], b.cnt[:k])
        assert torch.equal(a.stats, b.stats)
        assert torch.equal(a.ere[:k], b.ere[:k])
        assert torch.equal(a.g, b.g)
        assert int(a.ctr.item()) == int(b.ctr.item()) == 2


def _mixed(A):
    """Four problems of different models and sizes with their sample sets:
    BF16 MLP (h2o shape), FP32 MLP (small), BF16 transformer (6 orbitals),
    FP32 NADE (5 orbitals)."""
    from synthetic import flatten_nade, flatten_tf, integrals, nade_params, tf_params, workload
    out = []
    for name, form in (("h2o", "bf16"), ("small", "fp32")):
        w = workload(name, bias_std=0.2)
        ham = A.Hamiltonian(w["h"], w["g"], w["e_nuc"], w["n_alpha"], w["n_beta"])
        out.append((ham, A.Model.mlp(w["n"], w["width"], w["n_hidden"], torch.tensor(w["params"], device="cuda"),
                                     form)))
    h, g, e = integrals(21, 6, 6)
    ham = A.Hamiltonian(h, g, e, 3, 2)
    P = torch.tensor(flatten_tf(tf_params(21, 6, 64, 2, bias_std=0.2)), device="cuda")
    out.append((ham, A.Model.transformer(6, 64, 4, 2, P, "bf16")))
    h, g, e = integrals(22, 5, 5)
    ham = A.Hamiltonian(h, g, e, 2, 3)
    out.append((ham, A.Model.nade(5, 64, torch.tensor(flatten_nade(nade_params(22, 5, 64, bias_std=0.3)),
                                                      device="cuda"))))
    items = []
    for k, (ham, model) in enumerate(out):
        x, c = A.sample(model, ham, 50_000, seed=30 + k)
        items.append(dict(model=model, ham=ham, x=x, counts=c))
    return items


def test_batched_local_energy_equals_each_call_alone(A):
    """anqs_batched_local_energy runs each problem's anqs_local_energy on its
    own stream: the same kernels on the same inputs, so the results are the
    same bits; recorded in a CUDA graph and replayed, they are again."""
    items = _mixed(A)
    alone = [A.local_energy(it["model"], it["ham"], it["x"], it["counts"]) for it in items]
    batch = A.EnergyBatch(len(items))
    got = batch.local_energy(items)
    torch.cuda.synchronize()
    for (ar, ai, ast), (br, bi, bst) in zip(alone, got):
        assert torch.equal(ar, br) and torch.equal(ai, bi) and torch.equal(ast, bst)
    # the same call captured into a graph on a side stream, outputs cleared, replayed
    outs = [(torch.empty_like(r), torch.empty_like(i), torch.empty_like(st)) for r, i, st in alone]
    its = [dict(it, out=o) for it, o in zip(items, outs)]
    side = torch.cuda.Stream()
    side.wait_stream(torch.cuda.current_stream())
    graph = torch.cuda.CUDAGraph()
    with torch.cuda.stream(side):
        batch.local_energy(its, stream=side)  # workspaces allocated outside the capture
        ws = [batch._keep[3 * k + 2] for k in range(len(its))]
        its = [dict(it, workspace=w) for it, w in zip(its, ws)]
        torch.cuda.synchronize()
        with torch.cuda.graph(graph, stream=side):
            batch.local_energy(its, stream=side)
    for o in outs:
        for t in o:
            t.fill_(float("nan"))
    graph.replay()
    torch.cuda.synchronize()
    for (ar, ai, ast), (br, bi, bst) in zip(alone, outs):
        assert torch.equal(ar, br) and torch.equal(ai, bi) and torch.equal(ast, bst)


def test_batched_local_energy_checks_before_queueing(A):
    items = _mixed(A)[:3]
    outs = [(torch.full((it["x"].numel(),), float("nan"), dtype=torch.float64, device="cuda"),
             torch.full((it["x"].numel(),), float("nan"), dtype=torch.float64, device="cuda"),
             torch.full((4,), float("nan"), dtype=torch.float64, device="cuda")) for it in items]
    its = [dict(it, out=o) for it, o in zip(items, outs)]
    small = A.EnergyBatch(2)
    with pytest.raises(A.AnqsError, match="CAPACITY"):
        small.local_energy(its)
    batch = A.EnergyBatch(3)
    bad = dict(its[2], workspace=torch.empty(16, dtype=torch.uint8, device="cuda"))
    with pytest.raises(A.AnqsError, match="CAPACITY"):
        batch.local_energy(its[:2] + [bad])
    torch.cuda.synchronize()
    for o in outs:  # nothing of the failed calls ran
        assert all(torch.isnan(t).all() for t in o)


def _mlp_items(A, ks, n_samples=20_000):
    """16-bit MLP problems of the 32-problem workload (different orbital and
    electron counts, width 128) with their sample sets, plus one 16-bit MLP
    of width 64 (runs on its stream: the persistent launch takes one width)."""
    from synthetic import workload
    items = []
    for k in ks:
        p = batch32_problem(k)
        ham = A.Hamiltonian(p["h"], p["g"], p["e_nuc"], p["n_alpha"], p["n_beta"])
        params = torch.tensor(flatten_mlp(mlp_params(p["seed"], p["n"], p["width"], p["n_hidden"])), device="cuda")
        model = A.Model.mlp(p["n"], p["width"], p["n_hidden"], params, "bf16")
        x, c = A.sample(model, ham, n_samples, seed=40 + k)
        items.append(dict(model=model, ham=ham, x=x, counts=c))
    w = workload("small", bias_std=0.2)
    ham = A.Hamiltonian(w["h"], w["g"], w["e_nuc"], w["n_alpha"], w["n_beta"])
    model = A.Model.mlp(w["n"], w["width"], w["n_hidden"], torch.tensor(w["params"], device="cuda"), "bf16")
    x, c = A.sample(model, ham, 10_000, seed=3)
    items.insert(2, dict(model=model, ham=ham, x=x, counts=c))
    return items


def test_persistent_launch_every_schedule_equals_each_call_alone(A):
    """The persistent multi-problem launch computes every tile exactly as the
    single-problem launch does: for every schedule (static and dynamic, 4 to
    32 tiles per work item) and for plain streams, the local energies and
    statistics are the same bits as anqs_local_energy's."""
    from paper_2310_04166_gb300 import _lib
    items = _mlp_items(A, [0, 3, 5, 9, 14, 20, 27])
    alone = [A.local_energy(it["model"], it["ham"], it["x"], it["counts"]) for it in items]
    batch = A.EnergyBatch(len(items))
    assert batch.schedule == (_lib.ANQS_BATCH_DYNAMIC, 8)
    for mode in (_lib.ANQS_BATCH_STATIC, _lib.ANQS_BATCH_DYNAMIC, _lib.ANQS_BATCH_STREAMS):
        for chunk in (1, 3, 8, 32, 512):
            batch.set_schedule(mode, chunk)
            got = batch.local_energy(items)
            torch.cuda.synchronize()
            for (ar, ai, ast), (br, bi, bst) in zip(alone, got):
                assert torch.equal(ar, br) and torch.equal(ai, bi) and torch.equal(ast, bst), (mode, chunk)
    for it in items:
        assert it["model"].status() == 0


def test_autotune_keeps_the_fastest_schedule(A):
    from paper_2310_04166_gb300 import _lib
    items = _mlp_items(A, [1, 4, 8, 12])
    batch = A.EnergyBatch(len(items))
    times = batch.autotune(items)
    assert len(times) == 8 and all(t > 0 for t in times)
    mode, chunk = batch.schedule
    best = min(range(8), key=lambda i: times[i])
    assert (mode, chunk) == A.AUTOTUNE_CANDIDATES[best]
    alone = [A.local_energy(it["model"], it["ham"], it["x"], it["counts"]) for it in items]
    got = batch.local_energy(items)
    torch.cuda.synchronize()
    for (ar, ai, ast), (br, bi, bst) in zip(alone, got):
        assert torch.equal(ar, br) and torch.equal(ai, bi) and torch.equal(ast, bst)
    # refused while the stream is being captured (nothing is queued)
    side = torch.cuda.Stream()
    graph = torch.cuda.CUDAGraph()
    with torch.cuda.stream(side):
        with pytest.raises(A.AnqsError, match="capture"):
            with torch.cuda.graph(graph, stream=side):
                batch.autotune(items, stream=side)
    # no 16-bit MLP problem: nothing to tune
    w_items = [it for it in _mixed(A) if not (it["model"].desc.kind == _lib.ANQS_MODEL_MLP
                                              and it["model"].desc.form == _lib.ANQS_FORM_BF16)]
    with pytest.raises(A.AnqsError, match="UNSUPPORTED"):
        A.EnergyBatch(len(w_items)).autotune(w_items)


def test_batched_step_with_persistent_launch_equals_each_problem_alone(A):
    """The 32-problem workload's step shape (samplers on their streams, one
    batched local-energy call, gradients on their streams) in one CUDA graph
    gives every problem the pass it gets alone, bit for bit."""
    from paper_2310_04166_gb300.batch import BatchedStep
    ks = [2, 6, 11, 19, 23]
    batched = _problems(A, ks, "bf16", 20_000)
    alone = _problems(A, ks, "bf16", 20_000)
    bs = BatchedStep(batched, persistent=True)
    bs.eager()
    bs.autotune()
    bs.capture()
    bs.replay()
    for p in alone:
        for _ in range(3):
            p.step()
    torch.cuda.synchronize()
    for a, b in zip(batched, alone):
        k = int(a.nu.item())
        assert k == int(b.nu.item()) and k > 0
        assert torch.equal(a.x[:k], b.x[:k]) and torch.equal(a.cnt[:k], b.cnt[:k])
        assert torch.equal(a.stats, b.stats)
        assert torch.equal(a.ere[:k], b.ere[:k])
        assert torch.equal(a.g, b.g)
        assert int(a.ctr.item()) == int(b.ctr.item()) == 3


@pytest.mark.parametrize("fail_at", [1, 3])
def test_batched_local_energy_error_after_fork_joins_every_stream(A, fail_at, monkeypatch):
    """A problem that fails after its stream was forked (a host-side injected
    error, ANQS_BATCH_FAIL_AT): the call returns ANQS_ERR_CUDA, the problems
    queued before it complete, and the caller's stream is joined to every
    forked stream, eagerly and inside a CUDA-graph capture (which then ends
    without unjoined work)."""
    items = _mlp_items(A, [0, 3, 5], n_samples=10_000)  # 16-bit MLPs (persistent launch) and one width-64 MLP
    alone = [A.local_energy(it["model"], it["ham"], it["x"], it["counts"]) for it in items]
    outs = [(torch.full_like(r, float("nan")), torch.full_like(i, float("nan")), torch.full_like(st, float("nan")))
            for r, i, st in alone]
    its = [dict(it, out=o) for it, o in zip(items, outs)]
    batch = A.EnergyBatch(len(its))
    batch.set_schedule(_lib_mode(A, "streams"), 8)
    monkeypatch.setenv("ANQS_BATCH_FAIL_AT", str(fail_at))
    with pytest.raises(A.AnqsError, match="injected failure"):
        batch.local_energy(its)
    torch.cuda.synchronize()
    for k in range(fail_at):  # queued before the failure: complete and right
        assert torch.equal(outs[k][0], alone[k][0])
    # the persistent path: the failure stops the launch; nothing is left running
    batch.set_schedule(_lib_mode(A, "dynamic"), 8)
    with pytest.raises(A.AnqsError, match="injected failure"):
        batch.local_energy(its)
    torch.cuda.synchronize()
    # inside a capture: the error is raised, and the capture ends cleanly
    ws = [A._ws(A.local_energy_workspace_bytes(it["model"], it["ham"], it["x"].numel()), it["x"].device) for it in its]
    its_ws = [dict(it, workspace=w) for it, w in zip(its, ws)]
    side = torch.cuda.Stream()
    side.wait_stream(torch.cuda.current_stream())
    graph = torch.cuda.CUDAGraph()
    with torch.cuda.stream(side):
        with pytest.raises(A.AnqsError, match="injected failure"):
            with torch.cuda.graph(graph, stream=side):
                batch.local_energy(its_ws, stream=side)
    torch.cuda.synchronize()
    monkeypatch.delenv("ANQS_BATCH_FAIL_AT")
    got = batch.local_energy(its_ws)  # the handle still works
    torch.cuda.synchronize()
    for (ar, ai, ast), (br, bi, bst) in zip(alone, got):
        assert torch.equal(ar, br) and torch.equal(ai, bi) and torch.equal(ast, bst)


def _lib_mode(A, name):
    from paper_2310_04166_gb300 import _lib
    return {"streams": _lib.ANQS_BATCH_STREAMS, "static": _lib.ANQS_BATCH_STATIC,
            "dynamic": _lib.ANQS_BATCH_DYNAMIC}[name]
