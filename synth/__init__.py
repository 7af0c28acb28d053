"""Seeded synthetic lattices, operators and boundaries (input data only)."""
