"""Shared helpers for the GPU parity tests (CUDA path vs the FP64 oracle)."""
import numpy as np

# Tolerances.  FP64 path: energy within 1e-10 relative, forces within 1e-10
# of the RMS force (RMS over components).  Reduced forms (FP32 pair sums with
# double-float accumulation; split-BF16 fit): energy within 1e-6 relative and
# RMS force error within 1e-5 of the RMS force.
TOL = {
    "fp64": dict(energy=1e-10, force_rms=1e-10, force_max=1e-8, pot_rms=1e-10),
    "fp32": dict(energy=1e-6, force_rms=1e-5, force_max=1e-3, pot_rms=1e-6),
    "fp32_tc": dict(energy=1e-6, force_rms=1e-5, force_max=1e-3, pot_rms=1e-6),
}


def rms(a):
    a = np.asarray(a, dtype=np.float64)
    return float(np.sqrt(np.mean(a * a)))


def errors(gpu_F, ref_F, gpu_U=None, ref_U=None, gpu_pot=None, ref_pot=None):
    e = {}
    dF = np.asarray(gpu_F) - np.asarray(ref_F)
    e["force_rms"] = rms(dF) / rms(ref_F)
    e["force_max"] = float(np.abs(dF).max()) / rms(ref_F)
    if gpu_U is not None:
        e["energy"] = abs(gpu_U - ref_U) / abs(ref_U)
    if gpu_pot is not None:
        e["pot_rms"] = rms(np.asarray(gpu_pot) - np.asarray(ref_pot)) / rms(ref_pot)
    return e


def assert_within(e, prec, what=""):
    tol = TOL[prec]
    for k, v in e.items():
        assert v <= tol[k], f"{what} {prec}: {k} = {v:.3e} > {tol[k]:.1e}  (all: {e})"


def to_dev(*arrays):
    import torch
    return [torch.as_tensor(np.ascontiguousarray(a, dtype=np.float64)).cuda() for a in arrays]


# Self-image energy constant of a unit charge in a periodic cubic box of side
# L under conducting surroundings: U_self = XI q^2 / (2 L).
XI_CUBIC = -2.837297479


def energy_floor(q, L=1.0):
    """Energy scale of a periodic system below which |U| is a cancellation
    of much larger terms: 1/2 |XI| sum q^2 / L.  Relative energy errors use
    max(|U|, this) as the denominator."""
    return 0.5 * abs(XI_CUBIC) * float(np.sum(np.asarray(q) ** 2)) / L


def rel_energy_err(U, U_ref, q, L=1.0):
    return abs(U - U_ref) / max(abs(U_ref), energy_floor(q, L))
