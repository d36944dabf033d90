"""Skeleton -> constraint satisfaction problem, costs, gradients and Adam in FP64.

(Oracle; test infrastructure only.)

A skeleton is a list of actions (kind, box, surface).  Walking it with the
actions' preconditions and effects (Listing 1; appendix "Actions") gives the
continuous variables of one particle and the constraint / cost functions of
Sec. V-A:

  Pick(o, g, p, q)      con: Kin(q, o, g, p), Grasp(o, g), CFreeHold(o, g, q)
                        (+ joint limits of q, the Motion constraint's limit part)
  Place(o, g, p, s, q)  con: Kin(q, o, g, p), StablePlace(o, p, s),
                        CFreeHold(o, g, q), CFreePlace(o, p) (+ joint limits)
  MinimizeObjDist       cost: sum of pairwise distances of the moved boxes

With n_knots > 0 the motion between consecutive Pick/Place configurations is
a trajectory of n_knots knot configurations (Listing 1 MoveFree / MoveHold;
Sec. VIII, real-robot stacking: knot points, initialised by linear
interpolation between the start and end configurations):

  MoveFree(q1, q2, tau)        con: Motion(q1, tau, q2) (joint limits of every
                               knot), CFreeTraj(tau)  cost: TrajLength(tau)
  MoveHold(o, g, q1, q2, tau)  con: Motion, CFreeTrajHold(o, g, tau)
                               cost: TrajLength(tau)

With self_collision on, every configuration (knots included) also carries
SelfCollision: the CFree constraints' "does not cause robot self-collisions"
(appendix constraint definitions), tolerance 0 penetration (appendix
constraint tolerances).

The particle layout (Pick: grasp x,y,z,yaw then q; Place: placement x,y,yaw
then q) is the interface documented in include/tamp.h.

Readings of points the paper leaves open:
  * Kin is two constraints, translation (m) and rotation (geodesic angle, rad);
  * CFreeHold(o, g, q): arm spheres at q plus o's spheres held at FK(q) G(g)^-1,
    against the static cuboids and every other box at its current pose; the
    manipulated box o is not an obstacle for the arm at its own pick/place
    configurations;
  * CFreePlace(o, p): o's spheres at P(p) against the same environment;
  * a collision cost is the summed penetration depth max(0, r - sdf);
  * StablePlace: the box footprint's 4 corners, in the surface frame, each
    scored with the bound distance to the surface rectangle, summed; z is
    fixed by the surface (placements are x, y, yaw);
  * Grasp(o, g): bound distance of g_xyz to [-h_x, h_x] x [-h_y, h_y] x
    [h_z - 0.02, h_z], yaw free; with 6-DOF grasps (Sec. VIII setup: "top-down
    4-DOF or 6-DOF poses") g = (x, y, z, yaw, roll, pitch), G(g) =
    Trans(g) Rz(yaw) Ry(pitch) Rx(roll) Rx(pi), the position bounded by the
    whole box [-h, h] (the gripper may hold any side), the angles free;
  * knots: the knots of the motion into an action sit in the particle just
    before that action's own variables; CFreeTraj(Hold) is CFreeHold's
    penetration depth at each knot -- the arm, plus the held box on a MoveHold,
    against the static cuboids and every box not in the hand (on a MoveFree
    also the box about to be picked) -- checked at the knots only; TrajLength
    is the joint-space length sum_i ||w_{i+1} - w_i|| of the polyline q1,
    knots, q2; there is no motion before the first action (the scene has no
    initial configuration);
  * SelfCollision: the summed penetration max(0, r_a + r_b - ||c_a - c_b||)
    over the arm's sphere pairs of links i > j + 1 whose spheres do not
    already overlap at q = 0 (links that always touch are not a collision,
    like a robot's self-collision ignore list), plus the held box's spheres
    against links 0..n-2 (not the wrist and gripper that hold it).
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np
import torch

from . import geometry as G

DT = torch.float64
PICK, PLACE, GOAL = 0, 1, 2
KNOT = 2                                     # configuration kind of a trajectory knot

# term kinds (include/tamp.h: tamp_term_kind)
(KIN_POS, KIN_ROT, GRASP, STABLE_PLACE, CFREE_HOLD, CFREE_PLACE, JOINT_LIMIT, OBJ_DIST, CFREE_TRAJ,
 TRAJ_LEN, SELF_COLLISION) = range(11)
TERM_NAMES = ["kin_pos", "kin_rot", "grasp", "stable_place", "cfree_hold", "cfree_place",
              "joint_limit", "obj_dist", "cfree_traj", "traj_len", "self_collision"]
COST_KINDS = (OBJ_DIST, TRAJ_LEN)            # costs, never constraints (Eq. 3)


@dataclass
class Options:
    """Weights lambda_c and tolerances eps_c of Eq. 2 / Eq. 3 and Adam settings.

    Weights: all constraints 1.0 except the kinematic rotation error (5.0) and
    stable placement (2.0) (appendix "Cost Weights"); the goal weight 0.25 is
    the appendix's lambda for the object-distance cost.  Tolerances (appendix
    "Constraint Tolerances"): world collisions 1 mm, kinematics 5 mm / 0.05 rad,
    joint limits 0, containment 1 mm; grasp bounds 1 mm (reading).  Knots:
    CFreeTraj as the other collisions (1.0, 1 mm); TrajLength 0.01 per radian
    of joint-space path (reading: the paper gives no weight).  Self-collision:
    weight 1.0, tolerance 0 (appendix "Constraint Tolerances").
    """

    w: list = field(default_factory=lambda: [1.0, 5.0, 1.0, 2.0, 1.0, 1.0, 1.0, 0.25, 1.0, 0.01, 1.0])
    tol: list = field(default_factory=lambda: [5e-3, 0.05, 1e-3, 1e-3, 1e-3, 1e-3, 0.0, math.inf, 1e-3, math.inf,
                                               0.0])
    n_knots: int = 0                        # knot configurations per motion between actions
    grasp_dof: int = 4                      # 4: top-down (x, y, z, yaw); 6: + roll, pitch
    self_collision: bool = False            # SelfCollision term on every configuration
    lr_joint: float = 1e-2
    lr_pos: float = 3e-3
    lr_yaw: float = 1e-2
    beta1: float = 0.9
    beta2: float = 0.999
    eps: float = 1e-8
    optimize_grasp: bool = True
    scale_by_batch: bool = True


@dataclass
class Term:
    kind: int
    action: int            # index of the action that owns it
    box: int
    cfg: int = -1          # index of the q variable block (configuration), if any


class Problem:
    """The CSP induced by one skeleton on one scene."""

    def __init__(self, scene, actions, opts: Options | None = None):
        self.sc = scene
        self.opts = opts or Options()
        self.n = scene.n_joints
        self.actions = [tuple(int(v) for v in a) for a in actions]
        self.arm = dict(base=scene.base, tool=scene.tool, dh_a=scene.dh_a, dh_d=scene.dh_d,
                        dh_alpha=scene.dh_alpha, dh_offset=scene.dh_offset)
        self._self_pairs()
        self._walk()

    def _self_pairs(self):
        """Which link pairs SelfCollision tests: links i > j + 1 whose spheres
        do not overlap at q = 0; and the arm spheres the held box is tested
        against (links 0..n-2).  ``self.self_mask`` [S, S] marks the sphere
        pairs (a on the higher link), ``self.held_mask`` [S] the arm spheres."""
        sc, n = self.sc, self.n
        links = np.asarray(sc.sphere_link)
        S = links.size
        frames = G.forward_kinematics(self.arm, torch.zeros(1, n, dtype=DT))
        c0 = G.apply(frames[:, torch.as_tensor(links, dtype=torch.long)],
                     torch.as_tensor(sc.sphere_xyzr[:, :3], dtype=DT))[0].numpy()
        r = np.asarray(sc.sphere_xyzr[:, 3], dtype=np.float64)
        touch = np.linalg.norm(c0[:, None, :] - c0[None, :, :], axis=-1) < r[:, None] + r[None, :]
        self.self_links = set()
        for i in range(n + 1):
            for j in range(i - 1):
                if (links == i).any() and (links == j).any() and not touch[np.ix_(links == i, links == j)].any():
                    self.self_links.add((i, j))
        self.self_mask = np.zeros((S, S), dtype=bool)
        for a in range(S):
            for b in range(S):
                self.self_mask[a, b] = (int(links[a]), int(links[b])) in self.self_links
        self.held_mask = links <= n - 2

    # -------------------------------------------------------------- skeleton walk
    def _walk(self):
        """Assign variables and constraints by simulating the symbolic state."""
        B = self.sc.n_boxes
        pose = [("init",) for _ in range(B)]     # current pose source of each box
        held = None                              # (box, grasp offset) or None
        off = 0
        self.kinds = []                          # per component: 'q', 'gpos', 'gyaw', 'ppos', 'pyaw'
        self.configs = []                        # per configuration: dict
        self.terms: list[Term] = []
        self.goal_boxes = None
        self.segments = []                       # per motion: (first config, knot configs, last config, term)
        m = self.opts.n_knots
        for ai, (kind, b, s) in enumerate(self.actions):
            if kind in (PICK, PLACE) and m > 0 and self.configs:
                # the motion from the previous configuration into this action's
                hb = held[0] if held is not None else -1
                env = [(j, pose[j]) for j in range(B) if j != hb]
                knots = []
                for _ in range(m):
                    q_off = off
                    self.kinds += ["q"] * self.n
                    off += self.n
                    self.configs.append(dict(action=ai, kind=KNOT, box=hb, q_off=q_off,
                                             g_off=held[1] if held is not None else -1, env=env))
                    ci = len(self.configs) - 1
                    knots.append(ci)
                    for k in (CFREE_TRAJ, JOINT_LIMIT) + ((SELF_COLLISION,) if self.opts.self_collision else ()):
                        self.terms.append(Term(k, ai, hb, ci))
                prev = max(c for c, cf in enumerate(self.configs) if cf["kind"] != KNOT)
                self.terms.append(Term(TRAJ_LEN, ai, -1, len(self.segments)))
                self.segments.append(dict(start=prev, knots=knots, end=len(self.configs)))
            if kind == PICK:
                if held is not None:
                    raise ValueError(f"action {ai}: Pick while holding a box (HandEmpty fails)")
                if not (0 <= b < B) or pose[b][0] == "held":
                    raise ValueError(f"action {ai}: invalid box {b}")
                g_off = off
                self.kinds += ["gpos"] * 3 + ["gyaw"] + (["gyaw"] * 2 if self.opts.grasp_dof == 6 else [])
                off += self.opts.grasp_dof
                q_off = off
                self.kinds += ["q"] * self.n
                off += self.n
                env = [(j, pose[j]) for j in range(B) if j != b]
                cfg = dict(action=ai, kind=PICK, box=b, q_off=q_off, g_off=g_off,
                           target=pose[b], env=env)
                self.configs.append(cfg)
                ci = len(self.configs) - 1
                for k in (KIN_POS, KIN_ROT, GRASP, CFREE_HOLD, JOINT_LIMIT) + \
                        ((SELF_COLLISION,) if self.opts.self_collision else ()):
                    self.terms.append(Term(k, ai, b, ci))
                held = (b, g_off)
                pose[b] = ("held",)
            elif kind == PLACE:
                if held is None or held[0] != b:
                    raise ValueError(f"action {ai}: Place of a box that is not held")
                if not (0 <= s < self.sc.surf.shape[0]):
                    raise ValueError(f"action {ai}: invalid surface {s}")
                p_off = off
                self.kinds += ["ppos"] * 2 + ["pyaw"]
                off += 3
                q_off = off
                self.kinds += ["q"] * self.n
                off += self.n
                env = [(j, pose[j]) for j in range(B) if j != b]
                cfg = dict(action=ai, kind=PLACE, box=b, q_off=q_off, g_off=held[1],
                           target=("var", p_off, s), env=env)
                self.configs.append(cfg)
                ci = len(self.configs) - 1
                for k in (KIN_POS, KIN_ROT, STABLE_PLACE, CFREE_HOLD, CFREE_PLACE, JOINT_LIMIT) + \
                        ((SELF_COLLISION,) if self.opts.self_collision else ()):
                    self.terms.append(Term(k, ai, b, ci))
                pose[b] = ("var", p_off, s)
                held = None
            elif kind == GOAL:
                moved = [j for j in range(B) if pose[j][0] == "var"]
                self.goal_boxes = [(j, pose[j]) for j in moved]
                self.terms.append(Term(OBJ_DIST, ai, -1, -1))
            else:
                raise ValueError(f"action {ai}: unknown kind {kind}")
        self.D = off

    # -------------------------------------------------------------- helpers
    def _grasp(self, x, go, yaw=None):
        """G(g) of the grasp at component go (yaw replaced if given)."""
        y = x[:, go + 3] if yaw is None else yaw
        if self.opts.grasp_dof == 6:
            return G.grasp_pose6(x[:, go], x[:, go + 1], x[:, go + 2], y, x[:, go + 4], x[:, go + 5])
        return G.grasp_pose(x[:, go], x[:, go + 1], x[:, go + 2], y)

    def _grasp_bounds(self, b):
        h = self.sc.box_half[b]
        if self.opts.grasp_dof == 6:
            return (torch.tensor([-h[0], -h[1], -h[2]], dtype=DT), torch.tensor([h[0], h[1], h[2]], dtype=DT))
        return (torch.tensor([-h[0], -h[1], h[2] - 0.02], dtype=DT), torch.tensor([h[0], h[1], h[2]], dtype=DT))

    def _box_pose(self, src, b, x):
        """Pose of box b from its source: the scene's initial pose or a placement."""
        if src[0] == "init":
            bx, by, bz, byaw = (float(v) for v in self.sc.box_init[b])
            P = x.shape[0]
            return G.box_pose(*(torch.full((P,), v, dtype=DT) for v in (bx, by, bz, byaw)))
        _, p_off, s = src
        z = float(self.sc.surf[s, 5] + self.sc.box_half[b, 2])
        return G.box_pose(x[:, p_off], x[:, p_off + 1], torch.full_like(x[:, p_off], z), x[:, p_off + 2])

    def _box_spheres(self, b, T):
        loc = torch.as_tensor(self.sc.box_spheres[b], dtype=DT)   # [8,4]
        c = G.apply(T.unsqueeze(-3), loc[:, :3])                   # [P,8,3]
        return c, loc[:, 3]

    def _env_penetration(self, c, r, env, x):
        """Summed penetration of spheres (c [P,N,3], r [N]) into the environment."""
        P = x.shape[0]
        total = torch.zeros(P, dtype=DT)
        O = self.sc.obs_center.shape[0]
        for o in range(O):
            pen = G.sphere_box_penetration(c, r, torch.as_tensor(self.sc.obs_center[o], dtype=DT),
                                           torch.as_tensor(self.sc.obs_rot[o], dtype=DT),
                                           torch.as_tensor(self.sc.obs_half[o], dtype=DT))
            total = total + pen.sum(-1)
        for j, src in env:
            cj, rj = self._box_spheres(j, self._box_pose(src, j, x))         # [P,8,3]
            pen = G.sphere_sphere_penetration(c.unsqueeze(-2), r.view(-1, 1), cj.unsqueeze(-3), rj.view(1, -1))
            total = total + pen.sum((-1, -2))
        return total

    # -------------------------------------------------------------- Eq. 2 terms
    def term_values(self, x: torch.Tensor) -> torch.Tensor:
        """Unweighted J_c for every term, [P, n_terms] (FP64)."""
        sc = self.sc
        P = x.shape[0]
        out = [None] * len(self.terms)
        per_cfg = {}
        arm_c = torch.as_tensor(sc.sphere_xyzr[:, :3], dtype=DT)
        arm_r = torch.as_tensor(sc.sphere_xyzr[:, 3], dtype=DT)
        links = torch.as_tensor(sc.sphere_link, dtype=torch.long)
        for ci, cfg in enumerate(self.configs):
            q = x[:, cfg["q_off"]:cfg["q_off"] + self.n]
            frames = G.forward_kinematics(self.arm, q)                   # [P,n+1,4,4]
            ee = G.end_effector(self.arm, frames)
            jl = G.dist_from_bounds(q, torch.as_tensor(sc.q_lo, dtype=DT), torch.as_tensor(sc.q_hi, dtype=DT))
            if cfg["kind"] == KNOT:
                # CFreeTraj / CFreeTrajHold at this knot, and its joint limits (Motion)
                c_all = G.apply(frames[:, links], arm_c)
                r_all = arm_r
                if cfg["box"] >= 0:
                    Gp = self._grasp(x, cfg["g_off"])
                    held_c, held_r = self._box_spheres(cfg["box"], ee @ G.rigid_inverse(Gp))
                    c_all = torch.cat([c_all, held_c], dim=1)
                    r_all = torch.cat([arm_r, held_r])
                per_cfg[ci] = {CFREE_TRAJ: self._env_penetration(c_all, r_all, cfg["env"], x), JOINT_LIMIT: jl,
                               SELF_COLLISION: self._self_penetration(c_all, r_all)}
                continue
            g = x[:, cfg["g_off"]:cfg["g_off"] + 4]
            Gp = self._grasp(x, cfg["g_off"])
            b = cfg["box"]
            Tobj_target = self._box_pose(cfg["target"], b, x)
            e_pos, e_rot = G.pose_error(ee, Tobj_target @ Gp)
            # arm spheres in world, then the held box's spheres at FK(q) G(g)^-1
            arm_world = G.apply(frames[:, links], arm_c)                   # [P,S,3]
            held_c, held_r = self._box_spheres(b, ee @ G.rigid_inverse(Gp))
            c_all = torch.cat([arm_world, held_c], dim=1)
            r_all = torch.cat([arm_r, held_r])
            cfree_hold = self._env_penetration(c_all, r_all, cfg["env"], x)
            vals = {KIN_POS: e_pos, KIN_ROT: e_rot, CFREE_HOLD: cfree_hold, JOINT_LIMIT: jl,
                    SELF_COLLISION: self._self_penetration(c_all, r_all)}
            if cfg["kind"] == PICK:
                lo, hi = self._grasp_bounds(b)
                vals[GRASP] = G.dist_from_bounds(g[:, :3], lo, hi)
            else:
                _, p_off, s = cfg["target"]
                vals[STABLE_PLACE] = self._containment(b, s, x[:, p_off:p_off + 3])
                pc, pr = self._box_spheres(b, Tobj_target)
                vals[CFREE_PLACE] = self._env_penetration(pc, pr, cfg["env"], x)
            per_cfg[ci] = vals
        for ti, t in enumerate(self.terms):
            if t.kind == TRAJ_LEN:
                out[ti] = self._traj_length(self.segments[t.cfg], x)
            elif t.kind == OBJ_DIST:
                pos = torch.stack([self._box_pose(src, j, x)[:, :3, 3] for j, src in self.goal_boxes], dim=1) \
                    if self.goal_boxes else torch.zeros(P, 0, 3, dtype=DT)
                out[ti] = G.obj_dist(pos)
            else:
                out[ti] = per_cfg[t.cfg][t.kind]
        return torch.stack(out, dim=1) if out else torch.zeros(P, 0, dtype=DT)

    def _self_penetration(self, c, r):
        """SelfCollision of arm spheres c[:, :S] (then the held box's, if any)."""
        S = self.self_mask.shape[0]
        ca, ra = c[:, :S], r[:S]
        pen = G.sphere_sphere_penetration(ca.unsqueeze(-2), ra.view(-1, 1), ca.unsqueeze(-3), ra.view(1, -1))
        total = (pen * torch.as_tensor(self.self_mask, dtype=DT)).sum((-1, -2))
        if c.shape[1] > S:
            hc, hr = c[:, S:], r[S:]
            pen = G.sphere_sphere_penetration(hc.unsqueeze(-2), hr.view(-1, 1), ca.unsqueeze(-3), ra.view(1, -1))
            total = total + (pen * torch.as_tensor(self.held_mask, dtype=DT)).sum((-1, -2))
        return total

    def _waypoints(self, seg, x):
        cs = [seg["start"]] + seg["knots"] + [seg["end"]]
        return [x[:, self.configs[c]["q_off"]:self.configs[c]["q_off"] + self.n] for c in cs]

    def _traj_length(self, seg, x):
        """TrajLength: joint-space length of the polyline start, knots, end."""
        w = self._waypoints(seg, x)
        return sum(G.norm(w[i + 1] - w[i]) for i in range(len(w) - 1))

    def interpolate_knots(self, X):
        """Knot initialisation (Sec. VIII): each motion's knots evenly spaced on
        the straight joint-space line between its start and end
        configurations.  Returns a copy of X [P, D]."""
        x = np.array(X, dtype=np.float64)
        for seg in self.segments:
            qa = x[:, self.configs[seg["start"]]["q_off"]:self.configs[seg["start"]]["q_off"] + self.n]
            qb = x[:, self.configs[seg["end"]]["q_off"]:self.configs[seg["end"]]["q_off"] + self.n]
            m = len(seg["knots"])
            for j, c in enumerate(seg["knots"]):
                f = (j + 1) / (m + 1)
                o = self.configs[c]["q_off"]
                x[:, o:o + self.n] = qa + f * (qb - qa)
        return x

    def _containment(self, b, s, p):
        """StablePlace containment: sum over the footprint's 4 corners of the
        bound distance to the surface rectangle, in the surface frame."""
        cx, cy, syaw, hx, hy, _z = (float(v) for v in self.sc.surf[s])
        h = self.sc.box_half[b]
        cs, ss = math.cos(syaw), math.sin(syaw)
        c, si = torch.cos(p[:, 2]), torch.sin(p[:, 2])
        lo = torch.tensor([-hx, -hy], dtype=DT)
        hi = torch.tensor([hx, hy], dtype=DT)
        total = torch.zeros(p.shape[0], dtype=DT)
        for sx in (-1.0, 1.0):
            for sy in (-1.0, 1.0):
                wx = p[:, 0] + c * (sx * h[0]) - si * (sy * h[1])
                wy = p[:, 1] + si * (sx * h[0]) + c * (sy * h[1])
                dx, dy = wx - cx, wy - cy
                u = torch.stack([cs * dx + ss * dy, -ss * dx + cs * dy], dim=-1)
                total = total + G.dist_from_bounds(u, lo, hi)
        return total

    # -------------------------------------------------------------- Eq. 2 / 3 / 5
    def weights(self):
        return torch.tensor([self.opts.w[t.kind] for t in self.terms], dtype=DT)

    def tolerances(self):
        return torch.tensor([self.opts.tol[t.kind] for t in self.terms], dtype=DT)

    def constraint_mask(self):
        return torch.tensor([t.kind not in COST_KINDS for t in self.terms])

    def total_cost(self, x: torch.Tensor) -> torch.Tensor:
        """Eq. 2: J(x) = sum_c lambda_c J_c + sum_c' lambda_c' c'."""
        return (self.term_values(x) * self.weights()).sum(dim=1)

    def satisfied(self, terms: torch.Tensor) -> torch.Tensor:
        """Eq. 3: AND over constraints of J_c <= eps_c (costs never constrain)."""
        cm = self.constraint_mask()
        ok = terms[:, cm] <= self.tolerances()[cm]
        return ok.all(dim=1)

    def constraint_counts(self, terms: torch.Tensor) -> torch.Tensor:
        """Eq. 5 numerators: per constraint, number of particles with J_c <= eps_c."""
        cm = self.constraint_mask()
        return (terms[:, cm] <= self.tolerances()[cm]).sum(dim=0)

    def gradient(self, x: torch.Tensor):
        """(J [P], dJ/dx [P, D]) by reverse-mode differentiation of Eq. 2."""
        x = x.detach().clone().requires_grad_(True)
        J = self.total_cost(x)
        (g,) = torch.autograd.grad(J.sum(), x)
        return J.detach(), g

    # -------------------------------------------------------------- Adam (Sec. V-B)
    def learning_rates(self) -> torch.Tensor:
        o = self.opts
        lr = {"q": o.lr_joint, "gpos": o.lr_pos if o.optimize_grasp else 0.0,
              "gyaw": o.lr_yaw if o.optimize_grasp else 0.0, "ppos": o.lr_pos, "pyaw": o.lr_yaw}
        return torch.tensor([lr[k] for k in self.kinds], dtype=DT)

    def adam_step(self, x, m, v, t: int, grad, n_batch: int):
        """One Adam update (Kingma & Ba 2014, Algorithm 1) of the batch objective
        Eq. 4: the particle's gradient is scaled by 1/N_b.  ``t`` is the step
        number after the increment (1 for the first update)."""
        o = self.opts
        gsc = grad / n_batch if o.scale_by_batch else grad
        m = o.beta1 * m + (1.0 - o.beta1) * gsc
        v = o.beta2 * v + (1.0 - o.beta2) * gsc * gsc
        m_hat = m / (1.0 - o.beta1 ** t)
        v_hat = v / (1.0 - o.beta2 ** t)
        x = x - self.learning_rates() * m_hat / (torch.sqrt(v_hat) + o.eps)
        return x, m, v

    def optimize(self, x0, n_steps: int, m0=None, v0=None, t0: int = 0):
        """OptimizeParticles: Adam on Eq. 4 for n_steps.  Satisfaction (Eq. 3) is
        checked at x_t before each update and once more after the last one; the
        index of the first check with a satisfying particle is returned (-1 if
        none).

        Best satisfying record (Alg. 1 returns a satisfying particle; the
        soft-cost experiments keep the lowest-cost one): for each particle, among
        the checks k = 0..n_steps at which it satisfies Eq. 3, the state x_k of
        lowest Eq. 2 cost (the earliest of equal ones), with that cost and its
        check index t0 + k; best_iter -1 and best_cost +inf where it never
        satisfies."""
        x = torch.as_tensor(x0, dtype=DT).clone()
        P = x.shape[0]
        m = torch.zeros_like(x) if m0 is None else torch.as_tensor(m0, dtype=DT).clone()
        v = torch.zeros_like(x) if v0 is None else torch.as_tensor(v0, dtype=DT).clone()
        first = -1
        best_x = torch.zeros_like(x)
        best_cost = torch.full((P,), math.inf, dtype=DT)
        best_iter = torch.full((P,), -1, dtype=torch.long)

        def record(terms, k):
            sat = self.satisfied(terms)
            cost = (terms * self.weights()).sum(1)
            better = sat & (cost < best_cost)
            best_x[better] = x[better]
            best_cost[better] = cost[better]
            best_iter[better] = t0 + k

        for it in range(n_steps):
            with torch.no_grad():
                terms = self.term_values(x)
            if first < 0 and bool(self.satisfied(terms).any()):
                first = it
            record(terms, it)
            _, g = self.gradient(x)
            x, m, v = self.adam_step(x, m, v, t0 + it + 1, g, P)
        with torch.no_grad():
            terms = self.term_values(x)
        if first < 0 and bool(self.satisfied(terms).any()):
            first = n_steps
        record(terms, n_steps)
        return dict(x=x, m=m, v=v, terms=terms, first_iter=first,
                    satisfied=self.satisfied(terms), cost=(terms * self.weights()).sum(1),
                    best_x=best_x, best_cost=best_cost, best_iter=best_iter)

    # -------------------------------------------------------------- kink margins
    def kink_margin(self, x: torch.Tensor) -> torch.Tensor:
        """Per particle, the smallest distance (m or rad) of any quantity from a
        point where a cost's derivative jumps: a penetration switching on
        (r - sdf = 0), a bound being crossed, two box-frame axes tying for the
        inside distance, a norm at zero (pose errors, pair distances, the outside
        distance of an active pair), a rotation error at 0 or pi.  Parity tests
        exclude (and count) particles whose margin is below a threshold, because
        FP32 may land on the other side of such a point."""
        sc = self.sc
        P = x.shape[0]
        big = torch.full((P,), math.inf, dtype=DT)
        ms = [big]
        arm_c = torch.as_tensor(sc.sphere_xyzr[:, :3], dtype=DT)
        arm_r = torch.as_tensor(sc.sphere_xyzr[:, 3], dtype=DT)
        links = torch.as_tensor(sc.sphere_link, dtype=torch.long)
        lo_q = torch.as_tensor(sc.q_lo, dtype=DT)
        hi_q = torch.as_tensor(sc.q_hi, dtype=DT)

        def env_margins(c, r, env):
            out = []
            for o in range(sc.obs_center.shape[0]):
                R = torch.as_tensor(sc.obs_rot[o], dtype=DT)
                u = ((c - torch.as_tensor(sc.obs_center[o], dtype=DT)).unsqueeze(-2) @ R).squeeze(-2)
                qv = u.abs() - torch.as_tensor(sc.obs_half[o], dtype=DT)
                sdf = G.norm(qv.clamp(min=0.0)) + qv.amax(-1).clamp(max=0.0)
                gap = r - sdf
                out.append(gap.abs().amin(-1))
                near = gap > -1e-3
                srt = qv.sort(dim=-1, descending=True).values
                inside = srt[..., 0] < 0
                tie = torch.where(near & inside, srt[..., 0] - srt[..., 1], torch.full_like(gap, math.inf))
                onsurf = torch.where(near, sdf.abs(), torch.full_like(gap, math.inf))
                uz = torch.where(near.unsqueeze(-1) & (qv > -1e-3), u.abs(), torch.full_like(u, math.inf))
                out += [tie.amin(-1), onsurf.amin(-1), uz.amin((-1, -2))]
            for j, src in env:
                cj, rj = self._box_spheres(j, self._box_pose(src, j, x))
                d = G.norm(c.unsqueeze(-2) - cj.unsqueeze(-3))
                gap = r.view(-1, 1) + rj.view(1, -1) - d
                out.append(gap.abs().amin((-1, -2)))
                out.append(torch.where(gap > -1e-3, d, torch.full_like(d, math.inf)).amin((-1, -2)))
            return out

        def bound_margins(v, lo, hi):
            return [(v - lo).abs().amin(-1), (v - hi).abs().amin(-1)]

        def self_margins(c, r):
            if not self.opts.self_collision:
                return []
            S = self.self_mask.shape[0]
            out = []
            for cb, rb, mask in ((c[:, :S], r[:S], self.self_mask),
                                 (c[:, S:], r[S:], np.broadcast_to(self.held_mask, (c.shape[1] - S, S)))):
                if cb.shape[1] == 0:
                    continue
                d = G.norm(cb.unsqueeze(-2) - c[:, :S].unsqueeze(-3))
                gap = rb.view(-1, 1) + r[:S].view(1, -1) - d
                m = torch.as_tensor(np.ascontiguousarray(mask))
                inf = torch.full_like(d, math.inf)
                out.append(torch.where(m, gap.abs(), inf).amin((-1, -2)))
                out.append(torch.where(m & (gap > -1e-3), d, inf).amin((-1, -2)))
            return out

        for seg in self.segments:
            w = self._waypoints(seg, x)
            ms += [G.norm(w[i + 1] - w[i]) for i in range(len(w) - 1)]
        for cfg in self.configs:
            q = x[:, cfg["q_off"]:cfg["q_off"] + self.n]
            frames = G.forward_kinematics(self.arm, q)
            ee = G.end_effector(self.arm, frames)
            if cfg["kind"] == KNOT:
                c_all, r_all = G.apply(frames[:, links], arm_c), arm_r
                if cfg["box"] >= 0:
                    Gp = self._grasp(x, cfg["g_off"])
                    held_c, held_r = self._box_spheres(cfg["box"], ee @ G.rigid_inverse(Gp))
                    c_all, r_all = torch.cat([c_all, held_c], 1), torch.cat([arm_r, held_r])
                ms += env_margins(c_all, r_all, cfg["env"])
                ms += self_margins(c_all, r_all)
                ms += bound_margins(q, lo_q, hi_q)
                continue
            g = x[:, cfg["g_off"]:cfg["g_off"] + 4]
            Gp = self._grasp(x, cfg["g_off"])
            b = cfg["box"]
            Tt = self._box_pose(cfg["target"], b, x)
            e_pos, e_rot = G.pose_error(ee, Tt @ Gp)
            ms += [e_pos, e_rot, math.pi - e_rot]
            arm_world = G.apply(frames[:, links], arm_c)
            held_c, held_r = self._box_spheres(b, ee @ G.rigid_inverse(Gp))
            ms += env_margins(torch.cat([arm_world, held_c], 1), torch.cat([arm_r, held_r]), cfg["env"])
            ms += self_margins(torch.cat([arm_world, held_c], 1), torch.cat([arm_r, held_r]))
            ms += bound_margins(q, lo_q, hi_q)
            if cfg["kind"] == PICK:
                ms += bound_margins(g[:, :3], *self._grasp_bounds(b))
            else:
                _, p_off, s = cfg["target"]
                pc, pr = self._box_spheres(b, Tt)
                ms += env_margins(pc, pr, cfg["env"])
                cx, cy, syaw, hx, hy, _z = (float(v) for v in self.sc.surf[s])
                h = self.sc.box_half[b]
                p = x[:, p_off:p_off + 3]
                c, si = torch.cos(p[:, 2]), torch.sin(p[:, 2])
                cs, ss = math.cos(syaw), math.sin(syaw)
                for sx in (-1.0, 1.0):
                    for sy in (-1.0, 1.0):
                        wx = p[:, 0] + c * (sx * h[0]) - si * (sy * h[1]) - cx
                        wy = p[:, 1] + si * (sx * h[0]) + c * (sy * h[1]) - cy
                        u = torch.stack([cs * wx + ss * wy, -ss * wx + cs * wy], -1)
                        ms += bound_margins(u, torch.tensor([-hx, -hy], dtype=DT), torch.tensor([hx, hy], dtype=DT))
        if self.goal_boxes:
            pos = [self._box_pose(src, j, x)[:, :3, 3] for j, src in self.goal_boxes]
            for i in range(len(pos)):
                for j in range(i + 1, len(pos)):
                    ms.append(G.norm(pos[i] - pos[j]))
        return torch.stack(ms, 0).amin(0)
