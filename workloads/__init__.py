"""Seeded synthetic inputs shared by the CUDA path, the oracle and the benchmark.

This package holds only input generation: generating curves sampled at the
16 panel Gauss-Legendre points, material parameters and plane-wave
directions.  It contains none of the solver's arithmetic (no modal Green's
functions, no quadrature corrections, no assembly, no factorisation), so the
oracle and the CUDA path can both consume its output without sharing code.
"""
from .curves import Curve, sphere, cylinder, cone, random_body, torus, starfish, droplet, panel_nodes
from .configs import (Media, PlaneWave, Config, config_sphere, config_cylinder, config_random, config_batch,
                      config_pool,
                      plane_wave, paper_default_wave)

__all__ = ["Curve", "sphere", "cylinder", "cone", "random_body", "torus", "starfish", "droplet", "panel_nodes",
           "Media", "PlaneWave", "Config", "config_sphere", "config_cylinder",
           "config_random", "config_batch", "config_pool", "plane_wave", "paper_default_wave"]
