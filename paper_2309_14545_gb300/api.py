"""User-facing wrappers over the C ABI: a context owner and an autograd cost.

Still marshalling only -- every computation happens in libvp's kernels.
"""
from __future__ import annotations

import torch

from . import vp


class Validator:
    """Owns one vp_ctx with a robot and an environment loaded."""

    def __init__(self, robot, env, device: int = 0):
        self.device = int(device)
        self.ctx = vp.vp_create(self.device)
        self.dof = int(len(robot.joint_type))
        self.n_spheres = int(len(robot.sphere_radius))
        try:
            vp.vp_load_robot(self.ctx, robot)
            vp.vp_load_env(self.ctx, env)
        except Exception:
            vp.vp_destroy(self.ctx)
            self.ctx = None
            raise

    def close(self):
        if self.ctx is not None:
            vp.vp_destroy(self.ctx)
            self.ctx = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def _dev(self):
        return torch.device("cuda", self.device)

    def load_env(self, env):
        vp.vp_load_env(self.ctx, env)

    def fk_spheres(self, q, stream=None):
        out = torch.empty((q.shape[0], self.n_spheres, 3), dtype=torch.float32, device=self._dev())
        vp.vp_fk_spheres(self.ctx, q, out, stream)
        return out

    def validate_states(self, q, stream=None):
        out = torch.empty(q.shape[0], dtype=torch.uint8, device=self._dev())
        vp.vp_validate_states(self.ctx, q, out, stream)
        return out

    def edge_counts(self, q0, q1, resolution, stream=None):
        out = torch.empty(q0.shape[0], dtype=torch.int32, device=self._dev())
        vp.vp_edge_counts(self.ctx, q0, q1, float(resolution), out, stream)
        return out

    def validate_edges(self, q0, q1, counts=None, resolution=1.0 / 32.0, mode=vp.VP_MODE_PLAIN, stream=None,
                       out=None):
        if out is None:
            out = torch.empty(q0.shape[0], dtype=torch.uint8, device=self._dev())
        vp.vp_validate_edges(self.ctx, q0, q1, counts, float(resolution), out, mode, stream)
        return out

    def validate_edges_host(self, q0, q1, counts=None, resolution=1.0 / 32.0, mode=vp.VP_MODE_PLAIN, stream=None,
                            out=None):
        """Edge validation from host (CPU, ideally pinned) tensors, the copies
        overlapped with the work; returns the CPU uint8 verdicts, valid once
        `stream` has completed (synchronise it before reading)."""
        if out is None:
            out = torch.empty(q0.shape[0], dtype=torch.uint8, pin_memory=True)
        vp.vp_validate_edges_host(self.ctx, q0, q1, counts, float(resolution), out, mode, stream)
        return out

    def validate_edges_work(self, q0, q1, counts=None, resolution=1.0 / 32.0, mode=vp.VP_MODE_PLAIN, stream=None):
        out = torch.empty(q0.shape[0], dtype=torch.uint8, device=self._dev())
        work = torch.zeros(vp.VP_WORK_N, dtype=torch.int64, device=self._dev())
        vp.vp_validate_edges_work(self.ctx, q0, q1, counts, float(resolution), out, mode, work, stream)
        return out, work

    def autotune(self, q0, q1, counts=None, resolution=1.0 / 32.0, stream=None):
        vp.vp_autotune(self.ctx, q0, q1, counts, float(resolution), stream)

    def tiling(self):
        """Lanes per edge of each edge-length bucket (batched mode)."""
        return vp.vp_tiling(self.ctx)

    def set_tiling(self, lanes):
        """Pin the batched mode's lanes per edge, bucket by bucket."""
        vp.vp_set_tiling(self.ctx, lanes)

    def screen_rounds(self):
        """Screening rounds of the batched mode (0: single phase)."""
        return vp.vp_screen_rounds(self.ctx)

    def set_screen_rounds(self, rounds):
        vp.vp_set_screen_rounds(self.ctx, rounds)

    def check_order(self):
        """The check order: VP_ORDER_FREQUENT (4: the link pairs that
        collide most often first, links posed on demand),
        VP_ORDER_FREQUENT_TWO_PASS (5: the same in two passes over a batched
        call, the leading pairs of every edge first), or VP_ORDER_* bits: 1
        if primitives are checked before self pairs, plus 2 if each link is
        checked as soon as it is posed (else every link is posed first)."""
        return vp.vp_check_order(self.ctx)

    def set_check_order(self, order):
        vp.vp_set_check_order(self.ctx, order)

    def link_bounds(self):
        """(link spheres [L, 4], half spheres [L, 2, 4], half of each sphere
        [S]) as packed for the kernels, in each link's frame."""
        return vp.vp_link_bounds(self.ctx, self.dof + 1, self.n_spheres)

    def shortcut(self, paths, lengths, draws, resolution=1.0 / 32.0, stream=None):
        """Randomized shortcutting, in place on device tensors paths
        [P, W, D] float32 and lengths [P] int32, from draws [T, P, 2]."""
        vp.vp_shortcut_paths(self.ctx, paths, lengths, draws, resolution, stream)
        return paths, lengths

    def rrt_connect(self, start, goal, samples, range_=1.0, resolution=1.0 / 32.0, cap=1024, stream=None):
        """Batched RRT-Connect: one problem per row of start/goal [B, D],
        samples [B, T, D] (device float tensors).  Returns a dict of device
        tensors: status, iters, path [B, 2 cap, D], path_len, tree_sizes."""
        B, D = start.shape
        dev = self._dev()
        out = {"status": torch.empty(B, dtype=torch.int32, device=dev),
               "iters": torch.empty(B, dtype=torch.int32, device=dev),
               "path": torch.empty((B, 2 * cap, D), dtype=torch.float32, device=dev),
               "path_len": torch.empty(B, dtype=torch.int32, device=dev),
               "tree_sizes": torch.empty((B, 2), dtype=torch.int32, device=dev)}
        vp.vp_rrt_connect(self.ctx, start, goal, samples, range_, resolution, cap, out["status"], out["iters"],
                          out["path"], out["path_len"], out["tree_sizes"], stream)
        return out

    def fk_codegen(self, enable=True):
        """The FK kernel fk_spheres uses: True (1) the per-robot kernel
        generated and compiled at run time, False (0) the table-driven one,
        -1 automatic (the default: generated, else the table); returns the
        compile time in ms."""
        return vp.vp_fk_codegen(self.ctx, int(enable))

    def nearest(self, points, queries, stream=None):
        """(index int64 [N], squared distance float32 [N]) of each query's
        l2 nearest neighbour among the points (device float tensors)."""
        index = torch.empty(queries.shape[0], dtype=torch.int64, device=self._dev())
        dist2 = torch.empty(queries.shape[0], dtype=torch.float32, device=self._dev())
        vp.vp_nearest(self.ctx, points, queries, index, dist2, stream)
        return index, dist2

    def collision_cost(self, q, margin, grad=False, stream=None):
        cost = torch.empty(q.shape[0], dtype=torch.float32, device=self._dev())
        g = torch.empty_like(q) if grad else None
        vp.vp_collision_cost(self.ctx, q, float(margin), cost, g, stream)
        return (cost, g) if grad else cost

    def sync_status(self, stream=None):
        return vp.vp_sync_status(self.ctx, stream)

    def kernel_time(self, enable=True):
        """Enable/disable timing of the validation kernel; returns the last
        timed call's kernel milliseconds (-1 if none)."""
        return vp.vp_kernel_time(self.ctx, enable)


class CollisionCost(torch.autograd.Function):
    """c(q) = sum over robot spheres s and primitives o of
    max(0, r_s + margin - d(c_s, o))^2; backward runs the reverse-mode FK
    adjoint kernel (forward recomputed, then one backward sweep over joints)."""

    @staticmethod
    def forward(ctx, q, validator: Validator, margin: float):
        qc = q.detach().contiguous()
        cost, grad = validator.collision_cost(qc, margin, grad=True)
        ctx.save_for_backward(grad)
        return cost

    @staticmethod
    def backward(ctx, dcost):
        (grad,) = ctx.saved_tensors
        return grad * dcost[:, None], None, None


def path_validity(validator: Validator, paths, resolution=1.0 / 32.0, mode=vp.VP_MODE_BATCHED):
    """Boolean check of waypoint paths [P, W, D]: path p is valid iff all of
    its W-1 consecutive edges are valid at `resolution`."""
    P, W, D = paths.shape
    q0 = paths[:, :-1].reshape(-1, D).contiguous()
    q1 = paths[:, 1:].reshape(-1, D).contiguous()
    ok = validator.validate_edges(q0, q1, None, resolution, mode=mode)
    return ok.view(P, W - 1).bool().all(dim=1)


def repair_paths(validator: Validator, paths, margin=0.02, iters=100, lr=0.01, smooth=1.0,
                 resolution=1.0 / 32.0):
    """Push the interior waypoints of paths [P, W, D] out of collision by Adam
    on  sum_i c(q_i) + smooth * sum_i |q_{i+1} - 2 q_i + q_{i-1}|^2  (the
    cost and its gradient from the FK adjoint kernel; endpoints fixed), then
    re-judge every path with the boolean edge check.  A path the check
    accepted before and rejects after repair is kept as it was.

    Returns (paths, valid before [P], valid after [P]); the verdicts always
    come from the boolean check, never from the cost."""
    P, W, D = paths.shape
    before = path_validity(validator, paths, resolution)
    inner = paths[:, 1:-1].clone().requires_grad_(True)
    opt = torch.optim.Adam([inner], lr=lr)
    for _ in range(iters):
        opt.zero_grad()
        full = torch.cat([paths[:, :1], inner, paths[:, -1:]], dim=1)
        c = CollisionCost.apply(inner.reshape(-1, D), validator, margin).sum()
        acc = full[:, 2:] - 2 * full[:, 1:-1] + full[:, :-2]
        (c + smooth * (acc * acc).sum()).backward()
        opt.step()
    fixed = torch.cat([paths[:, :1], inner.detach(), paths[:, -1:]], dim=1).contiguous()
    ok_fixed = path_validity(validator, fixed, resolution)
    take = ok_fixed | ~before
    out = torch.where(take[:, None, None], fixed, paths).contiguous()
    return out, before, path_validity(validator, out, resolution)
