"""Seeded synthetic inputs: reaction mechanisms and cell fields.

This package is shared by the oracle tests, the GPU tests and the benchmark.  It only
draws inputs (species, stoichiometry, Arrhenius and thermo parameters, cell states
T, p, Y); it holds none of the chemistry arithmetic (no rates, no temperature
inversion, no integration, no density or energy evaluation).
"""
from .mechanism import h2_air_mechanism, hydrocarbon_mechanism, toy_mechanism, R_GAS, P_ATM
from .fields import (premix_mass_fractions, slab_field, sheet_field, amr_boxes, helix_box_fields,
                     surrogate_samples, stratified_sample)

__all__ = ["h2_air_mechanism", "hydrocarbon_mechanism", "toy_mechanism", "R_GAS", "P_ATM",
           "premix_mass_fractions", "slab_field", "sheet_field", "amr_boxes", "helix_box_fields",
           "surrogate_samples", "stratified_sample"]
