"""Velocity-model builder warps on the GPU (App. "Model builder modules"):
Squish (Alg. squish), Fault (Alg. fault) and a simplified Deposit
(Alg. deposit), for torch CUDA tensors of shape (nz, nx) or (nz, ny, nx).
Argument marshalling only: the warps run in libsim's kernels (sim_model_*
in include/sim.h). Every call returns new (velocity, label) tensors on the
input's device, so a generated model goes straight into Simulator /
set_model / batch."""
import numpy as np

from . import abi, sim_model_deposit, sim_model_fault, sim_model_squish


def _grid(v, lab):
    import torch
    if v.dim() not in (2, 3) or not v.is_cuda:
        raise ValueError("velocity must be a CUDA tensor of shape (nz, nx) or (nz, ny, nx)")
    v3 = v.detach().to(torch.float32).contiguous()
    if v3.dim() == 2:
        v3 = v3.unsqueeze(1)
    l3 = None
    if lab is not None:
        l3 = lab.detach().to(device=v.device, dtype=torch.int32).contiguous().reshape(v3.shape)
    return v3, l3


def _out(v, v3, l3):
    import torch
    vo = torch.empty_like(v3)
    lo = torch.empty_like(l3) if l3 is not None else None
    return vo, lo


def _shape_back(v, vo, lo):
    if v.dim() == 2:
        vo = vo.squeeze(1)
        lo = lo.squeeze(1) if lo is not None else None
    return vo, lo


def squish(v, lab, dz, fill=0.0, fill_label=-1):
    """Alg. squish: pull every column at z + dz (dz: (nx,) or (ny, nx) cells)."""
    import torch
    v3, l3 = _grid(v, lab)
    nz, ny, nx = v3.shape
    d = torch.as_tensor(dz, dtype=torch.float32, device=v.device).reshape(ny, nx).contiguous()
    vo, lo = _out(v, v3, l3)
    sim_model_squish(nz, ny, nx, v3, l3, d, fill, fill_label, vo, lo)
    return _shape_back(v, vo, lo)


def fault(v, lab, cz, cx, dip, radius, slip, direction=1, d_die=10.0, d_perp=1e9, theta_die=np.pi,
          azimuth=np.pi / 2, cy=0.0, fill=0.0, fill_label=-1):
    """Alg. fault (lengths in cells, angles in radians). The default azimuth
    pi/2 dips towards +x, the 2D case."""
    v3, l3 = _grid(v, lab)
    nz, ny, nx = v3.shape
    f = abi.SimFault(cz=cz, cy=cy, cx=cx, azimuth=azimuth, dip=dip, radius=radius, slip=slip,
                     direction=int(direction), pad=0, d_die=d_die, d_perp=d_perp, theta_die=theta_die)
    vo, lo = _out(v, v3, l3)
    sim_model_fault(nz, ny, nx, v3, l3, f, fill, fill_label, vo, lo)
    return _shape_back(v, vo, lo)


def deposit(v, lab, t, bounds, vbed, beta=0.0, a_eta=0.0, f_top=0.0, f_base=0.0, eta=None, offsets=None,
            label0=0):
    """Alg. deposit (simplified): lay a slab of t rows of beds on top of the
    model. bounds (nbeds - 1, [ny,] nx) bed boundary depths in rows; vbed
    (nbeds,) bed velocities; eta (nzt, [ny,] nx) texture or None; offsets
    (nbeds,) texture depth offsets (default 0)."""
    import torch
    v3, l3 = _grid(v, lab)
    nz, ny, nx = v3.shape
    vbed = np.asarray(vbed, np.float32)
    nb = len(vbed)
    b = None
    if nb > 1:
        b = torch.as_tensor(bounds, dtype=torch.float32, device=v.device).reshape(nb - 1, ny, nx).contiguous()
    e = None
    nzt = 1
    if eta is not None:
        e = torch.as_tensor(eta, dtype=torch.float32, device=v.device)
        nzt = e.shape[0]
        e = e.reshape(nzt, ny, nx).contiguous()
    off = np.zeros(nb, np.int32) if offsets is None else np.asarray(offsets, np.int32)
    p = abi.SimDeposit(t=int(t), nbeds=nb, nzt=nzt, label0=int(label0), beta=beta, a_eta=a_eta, f_top=f_top,
                       f_base=f_base)
    vo, lo = _out(v, v3, l3)
    sim_model_deposit(nz, ny, nx, v3, l3, p, b, vbed, off, e, vo, lo)
    return _shape_back(v, vo, lo)
