"""Time-step sensitivity of the layered-field iteration (the Δt study of Sec. 6).

The paper reports that results barely change for Δt between 0.1 and 5 and
that larger steps reach their goal in fewer iterations.  ``dt_sweep`` runs the
same seeds at several Δt through the library (every step and every label is
computed by the CUDA kernels) and reports, per Δt:

* ``steps_to_converge`` -- the step count after which no label changes any
  more within the run (labels are read every ``check_time`` units of
  simulated time, i.e. every max(1, round(check_time / Δt)) steps);
* ``agreement`` -- the fraction of vertices whose final label equals the
  label at the smallest Δt of the sweep;
* ``base_left`` -- vertices still labelled by the base layer at the end;
* ``ms`` -- device time of the whole run (steps and label reads).

Every Δt runs for the same simulated time ``horizon``, so the step count is
round(horizon / Δt).
"""
import time

import numpy as np

from . import _lib


def dt_sweep(V, F, seeds, dts=(0.1, 1.0, 5.0, 10.0), horizon=300.0, check_time=1.0, field_dtype="f32",
             params=None):
    params = dict(params or {})
    out = {}
    for dt in sorted(dts):
        steps = max(1, int(round(horizon / dt)))
        every = max(1, int(round(check_time / dt)))
        with _lib.Mesh(V, F, field_dtype=field_dtype, **dict(params, dt=float(dt))) as mesh:
            mesh.seed(seeds)
            t0 = time.perf_counter()
            done, last_change, prev = 0, 0, None
            while done < steps:
                n = min(every, steps - done)
                mesh.step(n)
                done += n
                lab = mesh.labels()
                if prev is None or not np.array_equal(lab, prev):
                    last_change = done
                prev = lab
            ms = 1e3 * (time.perf_counter() - t0)
            st = mesh.stats()
        out[float(dt)] = dict(steps=steps, check_every=every, steps_to_converge=last_change,
                              time_to_converge=last_change * float(dt), labels=prev,
                              base_left=int((prev == -1).sum()), skeleton_total=int(st["skeleton_total"]), ms=ms)
    ref = out[float(min(dts))]["labels"]
    for r in out.values():
        r["agreement"] = float(np.mean(r["labels"] == ref))
    return out
