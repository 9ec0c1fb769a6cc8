"""The bounds-checked build of the library (-DMP_CHECK_BOUNDS, built by
__graft_entry__.build() next to the product) on the small GPU cases: every
access of the MP loop to the planes, level-0 / level-1 keys, tiles, atom
list, top level, chunk and group lists is checked against its buffer, and a
failed check is reported by mp_run as an error naming the access site (the
access itself is skipped).  Each case must run clean and still match the
oracle under the strict parity rule.  The checked library is loaded in a
child process (one library per process)."""
import multiprocessing as mp

import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

if not torch.cuda.is_available():  # pragma: no cover - collected on CPU hosts too
    pytest.skip("needs a CUDA GPU", allow_module_level=True)


def _cases():
    from paper_2202_12380_gb300 import inputs
    b = inputs.blackman
    return [
        # (name, L list, dicts, eps, K, plan flags (2: MP_PEDANTIC, 4: MP_COEF_FP64),
        #  launch shape, resets every n selections)
        ("single", [8192], [(inputs.gauss_edge(256), 64, 256)], 1e-4, 300, 0, None, None),
        ("multi3 512x1", [16384], [(b(w), w // 4, w) for w in (128, 256, 512)], 1e-4, 300, 0,
         (512, 1), None),
        ("multi3 256x1", [16384], [(b(w), w // 4, w) for w in (128, 256, 512)], 1e-4, 300, 0,
         (256, 1), None),
        ("multi3 128x16", [16384], [(b(w), w // 4, w) for w in (128, 256, 512)], 1e-4, 300, 0,
         (128, 16), None),
        ("fig2 128x4", [4096], [(b(128), 64, 128), (inputs.hann(32), 16, 32)], 1e-4, 300, 0,
         (128, 4), None),
        ("mixed fp64 128x16", [12288], [(b(256), 64, 256), (inputs.gauss_edge(128), 32, 128),
                                        (inputs.hann(512), 128, 512)], 1e-4, 300, 4, (128, 16), None),
        ("mixed fp64 512x1", [12288], [(b(256), 64, 256), (inputs.gauss_edge(128), 32, 128),
                                       (inputs.hann(512), 128, 512)], 1e-4, 300, 4, (512, 1), None),
        ("pedantic", [16384], [(b(w), w // 4, w) for w in (128, 256, 512)], 1e-4, 200, 2, None, None),
        ("batch uneven", [2048, 8192, 4096, 16384, 3072], [(b(w), w // 4, w) for w in (128, 256, 512)],
         1e-4, 200, 0, None, None),
        # 6144 frames on one 128-thread CTA (cap 4096): grouped top level
        ("grouped top level", [1 << 17], [(b(128), 32, 128), (b(256), 64, 256)], 1e-4, 300, 0,
         (128, 1), None),
        ("resets", [16384], [(b(w), w // 4, w) for w in (128, 256, 512)], 1e-2, 300, 0, None, 60),
    ]


def _child(q):
    try:
        from oracle import cmp
        from paper_2202_12380_gb300 import build, inputs, mpgabor as mg
        from tests.parity import compare
        build.build(checked=True)  # no-op when __graft_entry__.build() made it
        mg.lib_path = lambda: build.LIB_CHECKED
        out = []
        for name, lens, dicts, eps, K, flags, shape, resets in _cases():
            xs = [inputs.as_f32(inputs.mixture(L, 500 + i, fs=16000.0)) for i, L in enumerate(lens)]
            plan = mg.mp_plan_create([g for g, _, _ in dicts], [a for _, a, _ in dicts],
                                     [M for _, _, M in dicts], eps, flags)
            st = mg.mp_analyze(plan, [torch.from_numpy(x).cuda() for x in xs])
            if shape:
                mg.mp_state_set_launch(st, *shape)
            if resets:
                mg.mp_state_set_resets(st, resets, 0.0)
            mg.mp_run(st, K, 200.0)  # raises MPError if a bounds check failed
            for bi, x in enumerate(xs):
                atoms, errs = mg.mp_get_atoms(st, bi), mg.mp_get_errors(st, bi)
                E0 = float(np.sum(x.astype(np.float64) ** 2))
                if resets:
                    ref = cmp.mp_coef_reset(dicts, x.astype(np.float64), eps, K, 200.0,
                                            reset_it=resets)
                else:
                    ref = cmp.mp_coef(dicts, x.astype(np.float64), eps, K, 200.0,
                                      pedantic=bool(flags & 2))
                r = compare(atoms, errs, E0, ref, min_checked=min(20, ref.n_atoms))
                out.append((name, bi, r["checked"]))
            st.close()
            plan.close()
        # the allocation-free entry point in the checked build
        dicts = [(inputs.blackman(w), w // 4, w) for w in (128, 256)]
        plan = mg.mp_plan_create([d[0] for d in dicts], [d[1] for d in dicts],
                                 [d[2] for d in dicts], 1e-4)
        x = torch.from_numpy(inputs.as_f32(inputs.mixture(8192, 600, fs=16000.0))).cuda()
        buf = torch.empty(200 * mg.ATOM_DTYPE.itemsize, dtype=torch.uint8, device="cuda")
        n, stop, snr = mg.mp_decompose_static(plan, x, 200, 200.0, buf, None)
        out.append(("static", 0, n))
        plan.close()
        q.put(("ok", out))
    except Exception as e:  # reported to the parent
        q.put(("error", repr(e)))


def test_bounds_checked_build_runs_clean_and_matches_oracle():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    p = ctx.Process(target=_child, args=(q,))
    p.start()
    status, payload = q.get(timeout=900)
    p.join(timeout=120)
    assert status == "ok", payload
    assert p.exitcode == 0
    names = {o[0] for o in payload}
    assert len(names) == len(_cases()) + 1
    print(payload)
