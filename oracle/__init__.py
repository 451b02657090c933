"""CPU oracle of the P-RSoXS forward model (test infrastructure only)."""
