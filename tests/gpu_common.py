"""Shared helpers of the GPU parity tests: matched (oracle, CUDA) grid pairs and
the seeded workloads. Inputs are generated once, on the oracle's nodes, by the
input module, and handed to both sides."""
import numpy as np
import torch

from oracle.transport import Grid as OGrid, Problem as OProblem
from paper_1104_5330_gb300 import inputs as I


def T():
    import paper_1104_5330_gb300.ts as ts
    return ts


def rel_l2(a, b):
    a = np.asarray(a, dtype=np.float64)
    b = np.asarray(b, dtype=np.float64)
    return float(np.linalg.norm((a - b).ravel()) / np.linalg.norm(b.ravel()))


def pair(R1, R2, Nr, Nt, Np, NT, NP, G=1, precision=0, scheme=0, bc=0, filter_on=False):
    og = OGrid(R1, R2, Nr, Nt, Np, NT, NP, groups=G)
    gg = T().Grid(R1, R2, Nr, Nt, Np, NT, NP, groups=G, precision=precision, scheme=scheme,
                  bc=bc, filter_on=filter_on)
    return og, gg


def cuda(a, dtype=torch.float64):
    return torch.as_tensor(np.ascontiguousarray(a), dtype=dtype, device="cuda")


def host(t):
    return t.detach().double().cpu().numpy()


def absorber_workload(og, seed=1104):
    """kappa = 1 + 0.5 sin(th) cos(ph), eta = kappa exp(-r^2), kappa_s = 0.5, seeded
    smooth F0 per group (seed + g), static inflow = F0 at the inflow nodes."""
    G = og.G
    kap, eta, ks = I.absorber_fields(og.r, og.theta, og.phi, groups=G)
    F0 = np.stack([I.seeded_smooth(og.r, og.theta, og.phi, og.Theta, og.Phi, seed + g, og.R1, og.R2)
                   for g in range(G)])
    gR1, gR2 = I.inflow_from(F0, og.NT)
    return kap, eta, ks, F0, gR1, gR2


def setup_both(og, gg, kap, eta, ks, gR1=None, gR2=None, scheme="rk4", bc="tau",
               filter_on=False):
    op = OProblem(og, kap, eta, ks, gR1, gR2, bc=bc, scheme=scheme, filter_on=filter_on)
    gg.set_coeffs(kap, eta, ks, gR1, gR2)
    return op
