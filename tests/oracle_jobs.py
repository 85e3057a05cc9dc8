"""Long oracle runs for the parity tests at the workloads' stated step counts.

The FP64 oracle needs minutes for these (1000 RK4 steps at N_r = 33, 100 steps
of the full 33 x 16^4 x 4-group workload, RK4 steps on the 65 x 32^4 grid, 50
steps of seeded problems of the 64-problem batch), so they are computed in
spawned worker processes, one per energy group (groups are independent), that
start when the test session has been collected and run while the other GPU
tests do. Each job writes its result to an .npy file and returns the path.

The workers call the oracle and the seeded input generators only; nothing here
touches the CUDA library. Every job rebuilds its inputs from the same seeds as
the GPU side of its test, one group at a time: the per-group fields of these
workloads are identical across groups (F0 seed = base seed + g).
"""
import os

# (name -> (function name, kwargs)); the test that uses a job names it
R = (0.2, 1.0)
C2_LONG = (33, 8, 8, 8, 8)          # N_r = 33 at the step count of the 4-group workload
C2_FULL = (33, 16, 16, 16, 16)
C3_FULL = (65, 32, 32, 32, 32)
C2_LONG_STEPS = 1000
C2_FULL_STEPS = 100
C3_STEPS = 2
C4_STEPS = 50
# seeded problems of the 64-problem batch (index into batch_problems(64, 1104)):
# 6: N_Theta = N_Phi = 24; 11: N_theta = 24; 1: N_Phi = 24; 13: N_r = 65
C4_PROBLEMS = (6, 11, 1, 13)


def _threads():
    for v in ("OMP_NUM_THREADS", "OPENBLAS_NUM_THREADS", "MKL_NUM_THREADS"):
        os.environ[v] = "1"


def _absorber_group(dims, g, seed=1104, summation="matrix"):
    from oracle.transport import Grid, Problem
    from paper_1104_5330_gb300 import inputs as I
    og = Grid(*R, *dims, groups=1, summation=summation)
    kap, eta, ks = I.absorber_fields(og.r, og.theta, og.phi, groups=1)
    F0 = I.seeded_smooth(og.r, og.theta, og.phi, og.Theta, og.Phi, seed + g, *R)[None]
    gR1, gR2 = I.inflow_from(F0, og.NT)
    return og, Problem(og, kap, eta, ks, gR1, gR2), F0


def absorber_steps(out, dims, g, nsteps, summation="matrix"):
    """Group g of the absorber workload after nsteps RK4 steps at dt = 0.4 h_min."""
    import numpy as np
    from paper_1104_5330_gb300 import inputs as I
    og, op, F0 = _absorber_group(dims, g, summation=summation)
    F = op.run(F0, I.dt_rule(*R, dims[0]), nsteps)
    np.save(out, F[0])
    return out


def batch_problem_steps(out, q, g, nsteps, scheme):
    """Group g of seeded batch problem q: kappa = s (1 + 0.5 sin th cos ph),
    eta = kappa exp(-r^2), kappa_s = 0.5, seeded smooth F0 (problem seed + g) with
    its inflow data, nsteps steps of `scheme` ("rk4" or "split") at the problem's
    dt = 0.4 h_min."""
    import dataclasses
    import numpy as np
    from oracle.transport import Grid, Problem
    from paper_1104_5330_gb300 import inputs as I
    s = I.batch_problems(64, 1104)[q]
    og = Grid(s.R1, s.R2, s.Nr, s.Ntheta, s.Nphi, s.NTheta, s.NPhi, groups=1)
    kap, eta, ks = I.batch_fields(dataclasses.replace(s, groups=1), og.r, og.theta, og.phi)
    F0 = I.seeded_smooth(og.r, og.theta, og.phi, og.Theta, og.Phi, s.seed + g, s.R1, s.R2)[None]
    gR1, gR2 = I.inflow_from(F0, og.NT)
    op = Problem(og, kap, eta, ks, gR1, gR2, scheme=scheme)
    F = op.run(F0, I.dt_rule(s.R1, s.R2, s.Nr), nsteps)
    np.save(out, F[0])
    return out


def jobs():
    """Every job: name -> (function, kwargs without `out`). Longest first."""
    from paper_1104_5330_gb300 import inputs as I
    J = {}
    for summ in ("matrix", "library"):
        J[f"c3/{summ}"] = (absorber_steps, dict(dims=C3_FULL, g=0, nsteps=C3_STEPS,
                                                 summation=summ))
    for g in range(4):
        J[f"c2full/g{g}"] = (absorber_steps, dict(dims=C2_FULL, g=g, nsteps=C2_FULL_STEPS))
    for summ in ("matrix", "library"):
        for g in range(2):
            J[f"c2long/{summ}/g{g}"] = (absorber_steps, dict(dims=C2_LONG, g=g,
                                                               nsteps=C2_LONG_STEPS,
                                                               summation=summ))
    specs = I.batch_problems(64, 1104)
    for scheme in ("rk4", "split"):
        for q in C4_PROBLEMS:
            for g in range(specs[q].groups):
                J[f"c4/{scheme}/p{q}/g{g}"] = (batch_problem_steps,
                                               dict(q=q, g=g, nsteps=C4_STEPS, scheme=scheme))
    return J


class Pool:
    """The running jobs: submitted at once to a spawn-started process pool."""

    def __init__(self, workdir, workers=None):
        import concurrent.futures as cf
        import multiprocessing as mp
        self.workdir = workdir
        n = workers or max(1, min(12, (os.cpu_count() or 2) - 2))
        self.ex = cf.ProcessPoolExecutor(max_workers=n, mp_context=mp.get_context("spawn"),
                                         initializer=_threads)
        self.fut = {}
        for name, (fn, kw) in jobs().items():
            out = os.path.join(workdir, name.replace("/", "_") + ".npy")
            self.fut[name] = self.ex.submit(fn, out=out, **kw)

    def result(self, name, timeout=1500):
        import numpy as np
        return np.load(self.fut[name].result(timeout=timeout))

    def close(self):
        for f in self.fut.values():
            f.cancel()
        self.ex.shutdown(wait=True, cancel_futures=True)
