"""Builders shared by the tests: turn a synthetic workload dict into an
oracle problem and (on a GPU) a library problem over the same FP32 values."""
import numpy as np


def oracle_problem(orc, d, **over):
    kw = dict(speed=d.get("speed"), current=d.get("current"), cost=d.get("cost"),
              h=d["h"], lam=d.get("lam", 1.0), v_out=d.get("v_out", 1.0),
              ntargets=d["ntargets"], periodic=d.get("periodic"), dyn=d.get("dyn", 0),
              dubins_v=d.get("dubins_v", 1.0), scale=d.get("scale"),
              controls_b=d.get("controls_b"), weights=d.get("weights", 0),
              interp=d.get("interp", 0))
    if d.get("log_speed") is not None:
        kw["speed"] = np.exp(np.asarray(d["log_speed"], dtype=np.float32).astype(np.float64))
    kw.update(over)
    return orc.Problem(d["shape"], d["lo"], d["hi"], d["controls"], d["labels"], **kw)


def gpu_problem(hjb, d, device="cuda", host=False, **over):
    import torch

    def t(a, dt=torch.float32):
        if a is None:
            return None
        a = np.ascontiguousarray(np.asarray(a))
        if host:
            return np.ascontiguousarray(a.astype({torch.float32: np.float32,
                                                  torch.uint8: np.uint8}[dt]))
        return torch.as_tensor(a).to(dt).to(device).contiguous()

    kw = dict(speed=t(d.get("speed")), current=t(d.get("current")), cost=t(d.get("cost")),
              log_speed=t(d.get("log_speed")), h=d["h"], lam=d.get("lam", 1.0),
              value_out=d.get("v_out", 1.0), n_targets=d["ntargets"],
              periodic=d.get("periodic"), dyn=d.get("dyn", 0), dubins_v=d.get("dubins_v", 1.0),
              scale=t(d.get("scale")), controls_b=d.get("controls_b"),
              weights=d.get("weights", 0), interp=d.get("interp", 0))
    kw.update(over)
    return hjb.Problem(d["shape"], d["lo"], d["hi"], np.asarray(d["controls"], np.float32),
                       t(d["labels"], torch.uint8), **kw)


def to_np(x):
    try:
        import torch
        if isinstance(x, torch.Tensor):
            return x.detach().cpu().numpy()
    except ImportError:
        pass
    return np.asarray(x)


def projection_reads(nk, r, coarse_nodes, shape):
    """Fine nodes (2D, grid shape (nx, ny)) whose projection through Con reads
    one of the given coarse nodes (a bool array over the nk[0] x nk[1] coarse
    grid): every fine node of a coarse cell that has such a vertex."""
    nx, ny = shape
    out = np.zeros((ny, nx), dtype=bool)
    for jy, jx in zip(*np.nonzero(np.asarray(coarse_nodes).reshape(nk[1], nk[0]))):
        for cy in (jy - 1, jy):
            for cx in (jx - 1, jx):
                if 0 <= cy <= nk[1] - 2 and 0 <= cx <= nk[0] - 2:
                    out[cy * r:cy * r + r + 1, cx * r:cx * r + r + 1] = True
    return out.reshape(-1)
