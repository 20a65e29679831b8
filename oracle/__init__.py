"""CPU oracle for the CGP Poisson path: test infrastructure, never on the product path."""
