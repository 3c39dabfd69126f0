"""Comparison helpers of the GPU parity tests (CUDA path against the FP64 oracle).

Binary64 bar: max|gpu - oracle| / max|oracle| <= 1e-12 per field and block. The kernels
perform the oracle's IEEE-rounded operations in its order, with the same stated cube-root
iteration, so the states agree bit for bit (test_gpu_parity_long checks that over a full
hour); the bar leaves room only for the budget sums, formed in another order.
Arrival times are threshold crossings of the maximum level, so a level that sits within
rounding of the threshold at some step may cross it one step apart in the two runs: such
cells must be rare, one step apart at most, and a cell that arrived in one run only must
have its maximum within rounding of the threshold.
Budget terms (outflow, clip, feedback) are sums of the same terms in another order:
1e-12 of the term, or of the block's volume where the term itself is a small remainder
of cancelling inflow and outflow.

Binary32 bar (the forecast bounds): max |eta error| <= 5 cm on open water (cells whose
3 x 3 neighbourhood is wet in both runs); at the moving shoreline the instantaneous level
of a cell that is wet in one run and just dry in the other differs by up to its water
depth, so there the forecast is held by the wet/dry mismatch (<= 0.5 % of cells) and the
maximum-height (inundation) error (<= 5 cm) instead; arrivals in one run only
<= 0.1 % of the cells that arrived; arrival error mean <= 1 step, max <= 10 steps.
"""
import numpy as np

TOL64 = 1e-12


def relerr(a, b):
    scale = np.abs(b).max()
    return np.abs(a - b).max() / scale if scale > 0 else np.abs(a - b).max()


def check_arrival(ga, oa, omax, dt, thr):
    diff = ga != oa
    assert diff.mean() <= 1e-4, diff.mean()
    both = diff & (ga >= 0) & (oa >= 0)
    assert np.all(np.abs(ga[both] - oa[both]) <= dt * (1 + 1e-9)), np.abs(ga[both] - oa[both]).max()
    one = (ga >= 0) != (oa >= 0)
    assert np.all(np.abs(omax[one] - thr) <= 1e-9), np.abs(omax[one] - thr).max()


def compare_fp64(h, o, nblocks, tol=TOL64, outputs=True, dt=None, thr=0.01, report=None):
    for k in range(nblocks):
        ge, gM, gN = h.get_state(k)
        oe, oM, oN = o.get_state(k)
        for name, a, b in (("eta", ge, oe), ("M", gM, oM), ("N", gN, oN)):
            e = relerr(a, b)
            if report is not None:
                report[name] = max(report.get(name, 0.0), e)
            assert e <= tol, (k, name, e)
        if outputs:
            gh, oh = h.max_height(k), o.max_height(k)
            assert np.array_equal(np.isnan(gh), np.isnan(oh)), k
            m = ~np.isnan(oh)
            if m.any():
                assert relerr(gh[m], oh[m]) <= tol
            check_arrival(h.arrival_time(k), o.arrival_time(k), np.where(m, oh, -np.inf),
                          o.dt if dt is None else dt, thr)
        gb, ob = h.budget(k), o.budget(k)
        V = abs(ob["volume"])
        assert abs(gb["volume"] - ob["volume"]) <= 1e-12 * V
        for key in ("outflow", "clip", "ring"):
            err = abs(gb[key] - ob[key])
            if report is not None:
                report["budget_" + key] = max(report.get("budget_" + key, 0.0),
                                              err / max(abs(ob[key]), 1e-300))
            assert err <= 1e-12 * max(abs(ob[key]), 1e-3 * V), (k, key, gb[key], ob[key])


def open_water(hb, e32, e64, dry_eps):
    """Cells whose 3 x 3 neighbourhood is wet in both runs (away from any shoreline)."""
    wet = (hb + e32 > dry_eps) & (hb + e64 > dry_eps)
    op = wet.copy()
    op[1:, :] &= wet[:-1, :]
    op[:-1, :] &= wet[1:, :]
    out = op.copy()
    out[:, 1:] &= op[:, :-1]
    out[:, :-1] &= op[:, 1:]
    return out


def fp32_metrics(h, o, sc):
    """Forecast-level differences of a binary32 handle from the oracle (or from a binary64
    handle): max |eta| error over all cells and over open water (m), max-height error
    (m), final wet/dry mismatch, arrival errors."""
    m = dict(eta=0.0, eta_open=0.0, maxh=0.0, wet_mis=0, cells=0, arr_mis=0, arrived=0,
             arr_err=[])
    for k in range(len(sc.blocks)):
        hb = np.asarray(sc.bathy[k])
        e32, e64 = h.get_state(k)[0], o.get_state(k)[0]
        d = np.abs(e32 - e64)
        m["eta"] = max(m["eta"], float(d.max()))
        ow = open_water(hb, e32, e64, sc.dry_eps)
        if ow.any():
            m["eta_open"] = max(m["eta_open"], float(d[ow].max()))
        g, r = h.max_height(k), o.max_height(k)
        both = ~np.isnan(g) & ~np.isnan(r)
        if both.any():
            m["maxh"] = max(m["maxh"], float(np.abs(g[both] - r[both]).max()))
        m["wet_mis"] += int(((hb + e32 > sc.dry_eps) != (hb + e64 > sc.dry_eps)).sum())
        m["cells"] += hb.size
        ga, ra = h.arrival_time(k), o.arrival_time(k)
        ab = (ga >= 0) & (ra >= 0)
        m["arr_err"].append(np.abs(ga[ab] - ra[ab]))
        m["arr_mis"] += int(((ga >= 0) != (ra >= 0)).sum())
        m["arrived"] += int((ra >= 0).sum())
    m["arr_err"] = np.concatenate(m["arr_err"])
    return m


def check_fp32(m, dt):
    """The forecast bounds of the binary32 path (module docstring)."""
    assert m["eta_open"] <= 0.05, m["eta_open"]
    assert m["maxh"] <= 0.05, m["maxh"]
    assert m["wet_mis"] <= 0.005 * m["cells"], m["wet_mis"]
    assert m["arr_mis"] <= 0.001 * max(m["arrived"], 1), m["arr_mis"]
    if m["arr_err"].size:
        assert m["arr_err"].mean() <= dt and m["arr_err"].max() <= 10 * dt
