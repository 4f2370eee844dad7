"""Density control of the Gaussian map on the GPU (include/gsr.h,
gsr_densify_adc, gsr_mcmc_relocate, gsr_mcmc_noise): argument marshalling
only.  Parameters are the planar torch tensors of render.PARAM_NAMES; every
random draw is an argument."""
from __future__ import annotations

from typing import Dict, Optional, Tuple

import torch

from . import binding as _b
from .render import PARAM_NAMES, gaussians_struct


def _stream() -> int:
    return torch.cuda.current_stream().cuda_stream


class DensityControl:
    """Adaptive density control and MCMC relocation / noise over one context."""

    def __init__(self, rast):
        self.ctx = rast.ctx
        self._ws: Optional[torch.Tensor] = None

    def _workspace(self, N: int, dev) -> torch.Tensor:
        need = self.ctx.density_workspace_size(N)
        if self._ws is None or self._ws.numel() < need or self._ws.device != torch.device(dev):
            self._ws = torch.empty(need, dtype=torch.uint8, device=dev)
        return self._ws

    @staticmethod
    def _outputs(params, cap: int):
        dev = params["means"].device
        out = {k: torch.empty((v.shape[0], cap) if v.dim() == 2 else (cap,), dtype=torch.float32, device=dev)
               for k, v in params.items()}
        s = _b.GaussiansOut(cap, *[out[k].data_ptr() for k in PARAM_NAMES])
        return out, s

    def densify_adc(self, params: Dict[str, torch.Tensor], sh_degree: int, grad, count, radius, split_normals,
                    grad_threshold: float, split_scale: float, min_opacity: float, max_screen_radius: float = 0.0,
                    max_world_scale: float = 0.0, capacity: Optional[int] = None,
                    sync: bool = True) -> Tuple[Dict[str, torch.Tensor], torch.Tensor]:
        """Returns (the new Gaussians, device int32 count).  split_normals:
        [2, 3, N] standard-normal draws.  With sync the arrays are cut to the
        count (one device sync); otherwise they have capacity columns (2 N by
        default) of which the first count are valid."""
        N = int(params["means"].shape[1])
        cap = 2 * N if capacity is None else int(capacity)
        g = gaussians_struct(*[params[k] for k in PARAM_NAMES], sh_degree)
        out, s = self._outputs(params, cap)
        n_out = torch.zeros(1, dtype=torch.int32, device=params["means"].device)
        ws = self._workspace(N, params["means"].device)
        prm = _b.AdcParams(grad_threshold, split_scale, min_opacity, max_screen_radius, max_world_scale)
        ptr = lambda t: 0 if t is None else t.data_ptr()
        st = self.ctx.densify_adc(g, ptr(grad), ptr(count), ptr(radius), ptr(split_normals), prm, s,
                                  n_out.data_ptr(), ws.data_ptr(), ws.numel(), _stream())
        self.ctx.check(st, "gsr_densify_adc")
        if sync:
            n = min(int(n_out.item()), cap)
            out = {k: (v[:, :n] if v.dim() == 2 else v[:n]).contiguous() for k, v in out.items()}
        return out, n_out

    def mcmc_relocate(self, params: Dict[str, torch.Tensor], sh_degree: int, draws: torch.Tensor,
                      min_opacity: float = 0.005) -> Tuple[Dict[str, torch.Tensor], torch.Tensor]:
        """draws: [N] uniform 32-bit integers (any 4-byte integer dtype, read as
        unsigned).  Returns (the relocated Gaussians, device int32 number of
        dead slots filled)."""
        N = int(params["means"].shape[1])
        if draws.element_size() != 4 or draws.numel() != N:
            raise ValueError("draws must hold N 4-byte integers")
        g = gaussians_struct(*[params[k] for k in PARAM_NAMES], sh_degree)
        out, s = self._outputs(params, N)
        moved = torch.zeros(1, dtype=torch.int32, device=params["means"].device)
        ws = self._workspace(N, params["means"].device)
        st = self.ctx.mcmc_relocate(g, draws.data_ptr(), min_opacity, s, moved.data_ptr(), ws.data_ptr(),
                                    ws.numel(), _stream())
        self.ctx.check(st, "gsr_mcmc_relocate")
        return out, moved

    def mcmc_noise(self, params: Dict[str, torch.Tensor], sh_degree: int, eta: torch.Tensor, scale: float,
                   means_out: Optional[torch.Tensor] = None) -> torch.Tensor:
        """New means [3, N] = mean + scale sigmoid(-100 (o - 0.005)) Sigma eta;
        means_out may be params["means"] (in place)."""
        g = gaussians_struct(*[params[k] for k in PARAM_NAMES], sh_degree)
        out = torch.empty_like(params["means"]) if means_out is None else means_out
        st = self.ctx.mcmc_noise(g, eta.data_ptr(), scale, out.data_ptr(), _stream())
        self.ctx.check(st, "gsr_mcmc_noise")
        return out
