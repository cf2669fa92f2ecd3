"""Error behaviour of the C ABI that needs no GPU: rec_init validates its
arguments before any CUDA call and reports the cause through rec_last_error;
the context-taking entry points reject a NULL context."""
import ctypes as C

import numpy as np
import pytest


def _init(params, box, n_boxes=1):
    from paper_2312_11448_gb300 import rec
    ctx = C.c_void_p()
    rc = rec.lib().rec_init(C.byref(params) if params is not None else None,
                            C.byref(box) if box is not None else None, n_boxes, None, C.byref(ctx))
    return rc, rec.lib().rec_last_error(None).decode(), ctx


def _box(n=8, n_packets=100, null=None, vel4=None):
    from paper_2312_11448_gb300 import rec
    fake = C.c_void_p(0x1000)  # never dereferenced: validation fails first
    f = {k: fake for k in ("delta", "vel4", "x_e", "T", "tally", "emis")}
    if null:
        f[null] = None
    if vel4 is not None:
        f["vel4"] = C.c_void_p(vel4)
    return rec.BoxDesc(n, f["delta"], f["vel4"], f["x_e"], f["T"], f["tally"], f["emis"], n_packets)


@pytest.mark.parametrize("bad,match", [
    (dict(h=-1.0), "cosmological"), (dict(Y_p=1.0), "cosmological"), (dict(L_box_kpc=0.0), "cosmological"),
    (dict(n_sub=0), "n_sub"), (dict(precision=7), "precision"), (dict(mixing=9), "mixing"),
    (dict(mixing=3, f_alpha=1.5), "f_alpha")])
def test_rec_init_rejects_bad_params(bad, match):
    from paper_2312_11448_gb300 import rec
    kw = {k: v for k, v in bad.items() if k not in ("n_sub", "precision", "mixing")}
    p, q = rec.make_params(**kw)
    for k in ("n_sub", "precision", "mixing"):
        if k in bad:
            setattr(p, k, bad[k])
    rc, msg, ctx = _init(p, _box())
    assert rc == rec.REC_EINVAL and match in msg and not ctx.value


@pytest.mark.parametrize("box_kw,match", [(dict(n=0), "box side"), (dict(n=1025), "box side"),
                                          (dict(null="tally"), "NULL"), (dict(n_packets=2 ** 32), "2^32"),
                                          (dict(vel4=0x1010), "32-byte aligned")])
def test_rec_init_rejects_bad_boxes(box_kw, match):
    from paper_2312_11448_gb300 import rec
    p, q = rec.make_params()
    rc, msg, ctx = _init(p, _box(**box_kw))
    assert rc == rec.REC_EINVAL and match in msg and not ctx.value


def test_rec_init_rejects_missing_arguments():
    from paper_2312_11448_gb300 import rec
    p, q = rec.make_params()
    rc, msg, _ = _init(None, _box())
    assert rc == rec.REC_EINVAL
    rc, msg, _ = _init(p, None)
    assert rc == rec.REC_EINVAL and "box" in msg
    bad_q = np.array([0.0, -1.0])  # decreasing emission profile table
    p2, _ = rec.make_params(quantiles=bad_q)
    rc, msg, _ = _init(p2, _box())
    assert rc == rec.REC_EINVAL and "emission profile" in msg


def test_null_context_is_rejected():
    from paper_2312_11448_gb300 import rec
    L = rec.lib()
    assert L.lya_scatter_mc(None, None, None, None, None) == rec.REC_EINVAL
    assert L.rec_step_trbdf2(None, 0, 1400.0, 1390.0, None) == rec.REC_EINVAL
    L.rec_free(None)  # NULL-safe
