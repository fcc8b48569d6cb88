"""Helpers for GPU tests: move numpy inputs to cuda:0 and run the library."""
import numpy as np
import torch

DEV = torch.device("cuda:0")


def to_dev(H, x0c=None, x0b=None):
    t = dict(eptr=torch.from_numpy(np.ascontiguousarray(H.eptr, dtype=np.int64)).to(DEV),
             pins=torch.from_numpy(np.ascontiguousarray(H.pins, dtype=np.int32)).to(DEV),
             w=torch.from_numpy(np.ascontiguousarray(H.w, dtype=np.float64)).to(DEV))
    if x0c is not None:
        t["x0c"] = torch.from_numpy(np.ascontiguousarray(x0c)).to(DEV)
        t["x0b"] = torch.from_numpy(np.ascontiguousarray(x0b)).to(DEV)
    return t


def run_pipeline(H, x0c, x0b, k, dtype, clique_mode=0, reduce=0):
    import paper_2511_06600_gb300 as hef
    t = to_dev(H, x0c, x0b)
    out = hef.hyperedge_resistance(H.n, t["eptr"], t["pins"], t["w"], t["x0c"], t["x0b"], k,
                                   dtype, clique_mode=clique_mode, reduce=reduce)
    torch.cuda.synchronize()
    return {key: (v.cpu().numpy() if torch.is_tensor(v) else v) for key, v in out.items()}


def rel_errors(R, ref):
    """Max relative error over scores >= 1e-3 max, p99 over all, normwise."""
    big = ref >= 1e-3 * ref.max()
    rel = np.abs(R - ref) / np.maximum(ref, 1e-300)
    return dict(max=float(rel[big].max()) if big.any() else 0.0,
                p99=float(np.percentile(rel[ref > 0], 99)) if (ref > 0).any() else 0.0,
                normwise=float(np.abs(R - ref).max() / max(ref.max(), 1e-300)))


def kendall_tau(a, b):
    from scipy.stats import kendalltau
    return float(kendalltau(a, b).statistic)
