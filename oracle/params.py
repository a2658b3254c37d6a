"""Derived constants of the scheme (oracle; test infrastructure only).

Eq. NS7: lambda = 3 sigma eta / (2 sqrt 2).
Eq. NS31: gamma0 = 3/2.
Eq. NS30: S/eta^2 >= sqrt(4 gamma0/(M lambda dt)); S = 0 on input selects the
  smallest admissible S (a reading: the paper gives only the inequality).
Eq. NS29: alpha = -S/(2 eta^2) (1 + sqrt(1 - 4 gamma0 eta^4/(M lambda dt S^2))).
NS26: c = alpha + S/eta^2 is the shift of the Psi solve.
After Eq. NS39: rho0 = min(rho1, rho2), nu_m >= 1/2 max(mu1, mu2)/min(rho1, rho2);
  nu_m = 0 on input selects equality.  mu1, mu2 are the solvent viscosities of
  Eq. NS9 (droplet solvent viscosity beta*mu1 when the droplet is viscoelastic).
"""
import math


class Derived:
    def __init__(self, prm: dict):
        p = dict(prm)
        self.dw = p.get("dw", 0.0)
        if self.dw < 0.0:
            raise ValueError("the wall relaxation D_w of Eq. NS15 must be >= 0")
        ag = p.get("alpha_giesekus", 0.0)
        if not (0.0 <= ag < 1.0):
            raise ValueError("the Giesekus mobility must lie in [0, 1)")
        self.p = p
        self.gamma0 = 1.5
        self.dt = p["dt"]
        self.kappa = self.dw * self.gamma0 / self.dt  # implicit wall coefficient of Eq. NS34
        self.eta = p["eta"]
        self.lam = 3.0 * p["sigma"] * p["eta"] / (2.0 * math.sqrt(2.0))
        self.mob = p["mobility"]
        self.Ml = self.mob * self.lam
        smin = self.eta ** 2 * math.sqrt(4.0 * self.gamma0 / (self.Ml * self.dt))
        S = p.get("S", 0.0) or smin
        if S < smin * (1.0 - 1e-12):
            raise ValueError("S violates Eq. NS30")
        disc = 1.0 - 4.0 * self.gamma0 * self.eta ** 4 / (self.Ml * self.dt * S * S)
        disc = max(disc, 0.0)
        self.S = S
        self.alpha = -S / (2.0 * self.eta ** 2) * (1.0 + math.sqrt(disc))
        self.c = self.alpha + S / self.eta ** 2
        # polymer.  Approach 2 of Eq. NS12 (polymer_approach 0, the default): constant
        # polymer parameters, the droplet phase viscoelastic, tau = (1 + phi)/2 tau_p.
        # Approach 1 (polymer_approach 1): mu_p, lambda_H and alpha linear in phi
        # (Eq. NS11) between the droplet's (mu_p1, wi, alpha_giesekus) and the
        # ambient's (mu_p2, wi2, alpha_giesekus2); tau = tau_p.
        self.approach1 = int(p.get("polymer_approach", 0)) == 1
        if int(p.get("polymer_approach", 0)) not in (0, 1):
            raise ValueError("polymer_approach must be 0 (Eq. NS12) or 1 (Eq. NS11)")
        if self.approach1:
            beta = p.get("beta", 1.0)
            self.mu_p2 = p.get("mu_p2", 0.0)
            self.visco = (beta < 1.0 and p["mu1"] > 0.0) or self.mu_p2 > 0.0
            if self.visco and not (p.get("wi", 0.0) > 0.0 and p.get("wi2", 0.0) > 0.0):
                raise ValueError("approach 1 needs both relaxation times wi, wi2 > 0")
            ag2 = p.get("alpha_giesekus2", 0.0)
            if not (0.0 <= ag2 < 1.0):
                raise ValueError("the Giesekus mobility must lie in [0, 1)")
            self.lam_h2 = p.get("wi2", 0.0)
            self.alpha_g2 = ag2
        else:
            self.visco = p.get("wi", 0.0) > 0.0 and p.get("beta", 1.0) < 1.0
            beta = p.get("beta", 1.0) if self.visco else 1.0
        self.mu_s1 = beta * p["mu1"]
        self.mu_p1 = (1.0 - beta) * p["mu1"]
        self.mu_s2 = p["mu2"]
        self.lam_h = p.get("wi", 0.0)
        self.alpha_g = ag  # Giesekus mobility (Eqs. NS18, NS22); 0 is Oldroyd-B
        # convective flux of the CH step: "central" (the GPU path's) or "weno5z" (the paper's)
        # convective flux of phi (CH) and Theta (LCR): "central" (0, the default) or
        # "weno5z" (1, the paper's scheme, Section 3.2.1 and before Eq. NS40)
        adv = p.get("advection", "central")
        self.advection = {0: "central", 1: "weno5z"}.get(adv, adv)
        if self.advection not in ("central", "weno5z"):
            raise ValueError("advection must be 'central' (0) or 'weno5z' (1)")
        self.rho1, self.rho2 = p["rho1"], p["rho2"]
        self.rho0 = min(self.rho1, self.rho2)
        self.nu_m = p.get("nu_m", 0.0) or 0.5 * max(self.mu_s1, self.mu_s2) / self.rho0
        self.cos_bot = math.cos(math.radians(p["theta_bot_deg"]))
        self.cos_top = math.cos(math.radians(p["theta_top_deg"]))
        self.uw_bot = p.get("uw_bot", 0.0)
        self.uw_top = p.get("uw_top", 0.0)
        self.g = (p.get("gx", 0.0), p.get("gy", 0.0), p.get("gz", 0.0))

    def rho(self, phi):
        """Eq. NS8 / dual3."""
        return 0.5 * (1.0 + phi) * self.rho1 + 0.5 * (1.0 - phi) * self.rho2

    def mu(self, phi):
        """Eq. NS9 / dual3 (solvent viscosity)."""
        return 0.5 * (1.0 + phi) * self.mu_s1 + 0.5 * (1.0 - phi) * self.mu_s2

    def polymer_props(self, phic):
        """(mu_p, lambda_H, alpha) at coarse centres: Eq. NS11 in approach 1, the
        droplet's constants in approach 2."""
        if not self.approach1:
            return self.mu_p1, self.lam_h, self.alpha_g
        a, b = 0.5 * (1.0 + phic), 0.5 * (1.0 - phic)
        return (a * self.mu_p1 + b * self.mu_p2, a * self.lam_h + b * self.lam_h2,
                a * self.alpha_g + b * self.alpha_g2)
